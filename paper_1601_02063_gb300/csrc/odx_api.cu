// Host side of the C ABI declared in include/odyssey.h: context and scratch management,
// argument validation, scene tables, launches, statistics and host-buffer rendering.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "kerr_device.cuh"
#include "odx_internal.h"

namespace odx {
}  // namespace odx

using namespace odx;

struct odx_ctx {
    int device = 0;
    int num_sms = 0;
    odx_launch launch{128, 3, 0, 2, 16};  // chunk 0 and persistent 2: each tracer's defaults
    unsigned long long *queue = nullptr;
    DevStats *stats = nullptr;
    DevScene *scenes = nullptr;
    int64_t scene_cap = 0;
    std::vector<DevScene> host_scenes;
    // buffers of odx_render_host
    cudaStream_t host_stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // device-to-host copies overlapping the next slab
    void *hbuf = nullptr;
    size_t hbuf_bytes = 0;
    std::string last_error;
    // scratch of odx_image_flux: plane table + chunk sums
    void *flux_buf = nullptr;
    size_t flux_bytes = 0;
    std::vector<unsigned char> host_planes;
    // optional per-launch timing of the tracing kernel
    bool time_kernels = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    size_t events_used = 0;
};

namespace {

const char *kVersion = "odyssey-gb300 0.1 (sm_103a)";

int32_t fail(odx_ctx *ctx, int32_t code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return code;
}

int32_t cuda_fail(odx_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, ODX_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define ODX_CUDA(ctx, call)                                            \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
    } while (0)

bool finite(double x) { return isfinite(x) != 0; }

int32_t validate_scene(odx_ctx *ctx, const odx_scene &s, int k, bool list_mode)
{
    if (!finite(s.a) || fabs(s.a) >= 1.0) return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: |a| must be < 1", k);
    const double rp = 1.0 + sqrt(1.0 - s.a * s.a);
    if (!finite(s.r_obs) || s.r_obs <= 10.0 * rp)
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: r_obs must exceed 10 r_+", k);
    if (!list_mode && (!finite(s.theta_obs) || s.theta_obs < 0.0 || s.theta_obs > M_PI))
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: theta_obs must lie in [0, pi]", k);
    if (!finite(s.phi_obs)) return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: phi_obs not finite", k);
    if (!list_mode) {
        if (!finite(s.alpha_min) || !finite(s.alpha_max) || !(s.alpha_min < s.alpha_max) ||
            !finite(s.beta_min) || !finite(s.beta_max) || !(s.beta_min < s.beta_max))
            return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: empty or non-finite window", k);
        if (s.n_alpha < 1 || s.n_beta < 1)
            return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: resolution must be >= 1", k);
    }
    if (s.emitter < ODX_EMIT_NONE || s.emitter > ODX_EMIT_SPOT)
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: unknown emitter %d", k, s.emitter);
    if (odx::disk_emitter(s.emitter) &&
        (!finite(s.r_in) || !finite(s.r_out) || !(s.r_out > 0.0) || !finite(s.q_emis)))
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: bad thin-disk parameters", k);
    if (s.emitter == ODX_EMIT_NT_DISK && (!(s.T0 > 0.0) || !finite(s.T0)))
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: NT disk needs T0 > 0", k);
    if (s.emitter == ODX_EMIT_TORUS || s.emitter == ODX_EMIT_NT_DISK ||
        s.emitter == ODX_EMIT_SYNCH || s.emitter == ODX_EMIT_SPOT) {
        if (s.n_freq < 1 || s.n_freq > ODX_MAX_FREQ)
            return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: n_freq must be 1..%d", k, ODX_MAX_FREQ);
        for (int f = 0; f < s.n_freq; ++f)
            if (!finite(s.freqs[f]) || !(s.freqs[f] > 0.0))
                return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: frequencies must be > 0", k);
    }
    if (s.emitter == ODX_EMIT_TORUS) {
        if (!finite(s.C_norm) || s.C_norm < 0.0 || !(s.theta_width > 0.0) || !(s.T0 > 0.0) ||
            !finite(s.ne_index) || !finite(s.T_index) || !finite(s.theta_width) || !finite(s.T0))
            return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: bad torus parameters", k);
    }
    if (s.emitter == ODX_EMIT_SYNCH) {
        if (!(s.n_e0 > 0.0) || !finite(s.n_e0) || !(s.beta_B > 0.0) || !finite(s.beta_B) ||
            !(s.mass > 0.0) || !finite(s.mass) || !(s.T0 > 0.0) || !finite(s.T0) ||
            !(s.theta_width > 0.0) || !finite(s.theta_width) || !finite(s.ne_index) ||
            !finite(s.T_index) || !finite(s.r_out) || !(s.r_out > 0.0))
            return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: bad synchrotron-shell parameters", k);
    }
    if (s.emitter == ODX_EMIT_SPOT) {
        if (!(s.spot_size > 0.0) || !finite(s.spot_size) || !finite(s.spot_r) ||
            !finite(s.spot_phase) || !finite(s.t_obs) || !(s.T0 > 0.0) || !finite(s.T0) ||
            !(s.C_norm >= 0.0) || !finite(s.C_norm))
            return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: bad hot-spot parameters", k);
    }
    if (!(s.rtol > 0.0) || !finite(s.rtol) || !(s.h0 > 0.0) || !finite(s.h0) ||
        !(s.hmax_frac > 0.0) || !finite(s.hmax_frac) || !(s.horizon_factor > 1.0) ||
        !finite(s.horizon_factor) || s.max_steps < 1)
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: bad integrator controls", k);
    if (s.convention != ODX_CONV_PHYSICAL && s.convention != ODX_CONV_LITERAL)
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: unknown convention", k);
    if (s.precision != ODX_FP64 && s.precision != ODX_MIXED)
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: unknown precision", k);
    if (s.precision == ODX_MIXED &&
        (!(s.rtol_fp32 > 0.0) || !finite(s.rtol_fp32) || !finite(s.r_switch) || s.r_switch < 0.0))
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: bad mixed-precision controls", k);
    if (s.rt_control != ODX_RT_CONTROLLED && s.rt_control != ODX_RT_RIDE)
        return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: unknown rt_control", k);
    return ODX_OK;
}

// Compiled transfer slots: 3 (the three-frequency workloads), 4 or 8.
int32_t nf_slots(int32_t emitter, int32_t n_freq)
{
    if (emitter != ODX_EMIT_TORUS && emitter != ODX_EMIT_SYNCH) return 0;
    return n_freq <= 3 ? 3 : (n_freq <= 4 ? 4 : 8);
}

int32_t ensure_scene_capacity(odx_ctx *ctx, int64_t n)
{
    if (n <= ctx->scene_cap) return ODX_OK;
    if (ctx->scenes) ODX_CUDA(ctx, cudaFree(ctx->scenes));
    ctx->scenes = nullptr;
    ctx->scene_cap = 0;
    const int64_t cap = n < 64 ? 64 : n;
    ODX_CUDA(ctx, cudaMalloc(&ctx->scenes, cap * sizeof(DevScene)));
    ctx->scene_cap = cap;
    return ODX_OK;
}

int32_t set_device(odx_ctx *ctx)
{
    ODX_CUDA(ctx, cudaSetDevice(ctx->device));
    return ODX_OK;
}

// Event pair for timing the next tracing-kernel launch (none when timing is off or the
// stream is being captured).
void timing_events(odx_ctx *ctx, cudaStream_t st, cudaEvent_t *e0, cudaEvent_t *e1)
{
    *e0 = *e1 = nullptr;
    if (!ctx->time_kernels) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (ctx->events_used == ctx->events.size()) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
        ctx->events.push_back({a, b});
    }
    *e0 = ctx->events[ctx->events_used].first;
    *e1 = ctx->events[ctx->events_used].second;
    ++ctx->events_used;
}

// Validate, build the scene table, copy it and launch.  Shared by the render and list paths.
int32_t submit(odx_ctx *ctx, const odx_scene *scenes, int32_t n_scenes, const double *rays,
               int64_t n_list, odx_ray_record *records, double *image, cudaStream_t st,
               int64_t *total_rays, int64_t *total_image, int64_t id_begin = 0,
               int64_t id_end = 0)
{
    const bool list_mode = rays != nullptr || n_list >= 0;
    if (!scenes || n_scenes < 1) return fail(ctx, ODX_ERR_INVALID_ARG, "no scenes");
    if (!records) return fail(ctx, ODX_ERR_INVALID_ARG, "records pointer is NULL");
    if (((uintptr_t)records & 15u) != 0)
        return fail(ctx, ODX_ERR_INVALID_ARG, "records must be 16-byte aligned");
    if (image && ((uintptr_t)image & 7u) != 0)
        return fail(ctx, ODX_ERR_INVALID_ARG, "image must be 8-byte aligned");
    for (int k = 0; k < n_scenes; ++k) {
        int32_t rc = validate_scene(ctx, scenes[k], k, list_mode);
        if (rc != ODX_OK) return rc;
        if (scenes[k].emitter != scenes[0].emitter || scenes[k].precision != scenes[0].precision ||
            odx::scene_planes(scenes[k]) != odx::scene_planes(scenes[0]))
            return fail(ctx, ODX_ERR_INVALID_ARG,
                        "scene %d: all scenes of one call must share emitter, precision, n_freq", k);
    }
    ctx->host_scenes.resize(n_scenes);
    int64_t ray = 0, img = 0;
    const int64_t nf = odx::scene_planes(scenes[0]);
    for (int k = 0; k < n_scenes; ++k) {
        DevScene &d = ctx->host_scenes[k];
        const int64_t nk = list_mode ? n_list : (int64_t)scenes[k].n_alpha * scenes[k].n_beta;
        fill_dev_scene(d, scenes[k], ray, nk, img);
        ray += nk;
        img += nf * nk;
    }
    if (total_rays) *total_rays = ray;
    if (total_image) *total_image = img;
    if (list_mode && n_list > 0 && !rays)
        return fail(ctx, ODX_ERR_INVALID_ARG, "rays pointer is NULL");
    if (ray == 0) return ODX_OK;
    int32_t rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    rc = ensure_scene_capacity(ctx, n_scenes);
    if (rc != ODX_OK) return rc;
    ODX_CUDA(ctx, cudaMemcpyAsync(ctx->scenes, ctx->host_scenes.data(),
                                  n_scenes * sizeof(DevScene), cudaMemcpyHostToDevice, st));
    ODX_CUDA(ctx, cudaMemsetAsync(ctx->queue, 0, sizeof(unsigned long long), st));
    TraceArgs a{};
    a.scenes = ctx->scenes;
    a.n_scenes = n_scenes;
    a.list_mode = list_mode ? 1 : 0;
    a.rays = rays;
    a.n_total = ray;
    a.id_begin = id_begin;  // a slab of the render (both 0: every ray)
    a.id_end = id_end;
    a.records = records;
    a.image = image;
    a.queue = ctx->queue;
    a.stats = ctx->stats;
    a.chunk = ctx->launch.chunk;
    a.persistent = ctx->launch.persistent;
    a.fp64_batch = ctx->launch.fp64_batch;
    set_launch_medium(a, ctx->host_scenes[0],
                      list_mode || shared_medium(ctx->host_scenes.data(), n_scenes));
    const int32_t slots = nf_slots(scenes[0].emitter, scenes[0].n_freq);
    cudaEvent_t ev0, ev1;
    timing_events(ctx, st, &ev0, &ev1);
    cudaError_t e = scenes[0].precision == ODX_MIXED
                        ? launch_trace_mixed(a, slots, ctx->launch, ctx->num_sms, st, ev0, ev1)
                        : launch_trace_fp64(a, slots, ctx->launch, ctx->num_sms, st, ev0, ev1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trace kernel launch");
    return ODX_OK;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Launch the tracer over a scene table already resident on the device (graph capture).
int32_t launch_resident(odx_ctx *ctx, const DevScene *dev_table, const DevScene *host_table,
                        const odx_scene *scenes, int32_t n_scenes, int64_t n_total,
                        odx_ray_record *records, double *image, cudaStream_t st)
{
    ODX_CUDA(ctx, cudaMemsetAsync(ctx->queue, 0, sizeof(unsigned long long), st));
    TraceArgs a{};
    a.scenes = dev_table;
    a.n_scenes = n_scenes;
    a.list_mode = 0;
    a.rays = nullptr;
    a.n_total = n_total;
    a.records = records;
    a.image = image;
    a.queue = ctx->queue;
    a.stats = ctx->stats;
    a.chunk = ctx->launch.chunk;
    a.persistent = ctx->launch.persistent;
    a.fp64_batch = ctx->launch.fp64_batch;
    set_launch_medium(a, host_table[0], shared_medium(host_table, n_scenes));
    const int32_t slots = nf_slots(scenes[0].emitter, scenes[0].n_freq);
    cudaEvent_t ev0, ev1;
    timing_events(ctx, st, &ev0, &ev1);
    cudaError_t e = scenes[0].precision == ODX_MIXED
                        ? launch_trace_mixed(a, slots, ctx->launch, ctx->num_sms, st, ev0, ev1)
                        : launch_trace_fp64(a, slots, ctx->launch, ctx->num_sms, st, ev0, ev1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trace kernel launch");
    return ODX_OK;
}

}  // namespace

struct odx_graph {
    odx_ctx *ctx = nullptr;
    DevScene *table = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace odx {
void fill_dev_scene(DevScene &d, const odx_scene &s, int64_t ray_begin, int64_t n_rays,
                    int64_t img_offset)
{
    memset(&d, 0, sizeof(d));
    d.s = s;
    d.ray_begin = ray_begin;
    d.n_rays = n_rays;
    d.img_offset = img_offset;
    d.o_sto = sin(s.theta_obs);
    d.o_cto = cos(s.theta_obs);
    d.o_spo = sin(s.phi_obs);
    d.o_cpo = cos(s.phi_obs);
    d.o_Ro = sqrt(s.r_obs * s.r_obs + s.a * s.a);
    d.o_r_isco = isco_radius(s.a);
    d.o_r_stop = s.horizon_factor * horizon_radius(s.a);
    d.f_r_out = (float)s.r_out;
    d.f_hmax_frac = (float)s.hmax_frac;
    d.f_rtol32 = (float)s.rtol_fp32;
    // torus (Section 4.2): n_e^2 = r^(-2 ne_index) exp(-cos^2 / w^2), T_e = T0 r^-T_index
    const bool torus = s.emitter == ODX_EMIT_TORUS && s.T0 > 0.0 && s.theta_width > 0.0;
    d.f_T_index = (float)s.T_index;
    d.f_inv_T0 = torus ? (float)(1.0 / s.T0) : 0.f;
    d.f_lr_pref = (float)(0.5 * s.T_index - 2.0 * s.ne_index);
    d.f_c2_pref = torus ? (float)(-1.0 / (s.theta_width * s.theta_width)) : 0.f;
    d.f_pref0 = torus ? (float)(s.C_norm / sqrt(s.T0)) : 0.f;
    // synchrotron shell (Section 4.5): n_e / n_e0 = r^-ne_index exp(-cos^2 / (2 w^2)),
    // 1 / Theta_e = r^T_index / T0, frequencies in GHz
    const bool synch = s.emitter == ODX_EMIT_SYNCH && s.T0 > 0.0 && s.theta_width > 0.0 &&
                       s.n_e0 > 0.0 && s.beta_B > 0.0 && s.mass > 0.0;
    if (synch) {
        const SynchK q = synch_constants(s);
        d.f_synch = 1;
        d.f_inv_T0 = (float)(1.0 / s.T0);
        d.f_lr_pref = (float)(-s.ne_index);
        d.f_c2_pref = (float)(-1.0 / (2.0 * s.theta_width * s.theta_width));
        d.f_inv_kc = (float)q.inv_kc;
        d.f_ky = (float)q.ky;
        d.f_Atau = (float)q.Atau;
    }
    if (s.emitter == ODX_EMIT_SPOT) {
        const double rs = spot_orbit_radius(s), om = spot_omega(s);
        const double two_pi = 6.283185307179586;
        d.f_spot_Rs = (float)sqrt(rs * rs + s.a * s.a);
        d.f_spot_om = (float)om;
        d.f_spot_ph = (float)(s.spot_phase + om * s.t_obs - two_pi * floor((s.spot_phase + om * s.t_obs) / two_pi));
        d.f_spot_R4 = (float)(4.0 * s.spot_size);
    }
    const double nu_scale = synch ? 1.0 / kNuUnit : 1.0;
    const int nf = (s.n_freq > 0 && s.n_freq <= ODX_MAX_FREQ) ? s.n_freq : 0;
    for (int k = 0; k < ODX_MAX_FREQ; ++k) {
        const double nu = nf > 0 ? s.freqs[k < nf ? k : nf - 1] * nu_scale : 1.0;
        d.f_nu[k] = (float)nu;
        d.f_inv_nu3[k] = (nu > 0.0) ? (float)(1.0 / (nu * nu * nu)) : 0.f;
        d.rt_floor[k] = (nf > 0 && (s.emitter == ODX_EMIT_TORUS || synch))
                            ? rt_floor(s, s.freqs[k < nf ? k : nf - 1])
                            : INFINITY;
        d.f_rt_floor[k] = (float)d.rt_floor[k];
    }
}

static_assert(sizeof(MedConst) == (11 + 3 * ODX_MAX_FREQ) * 4, "MedConst has no padding");

static MedConst medium_const(const DevScene &d)
{
    MedConst m;
    m.T_index = d.f_T_index;
    m.inv_T0 = d.f_inv_T0;
    m.lr_pref = d.f_lr_pref;
    m.c2_pref = d.f_c2_pref;
    m.pref0 = d.f_pref0;
    for (int k = 0; k < ODX_MAX_FREQ; ++k) {
        m.nu[k] = d.f_nu[k];
        m.inv_nu3[k] = d.f_inv_nu3[k];
        m.rt_floor[k] = d.f_rt_floor[k];
    }
    m.inv_kc = d.f_inv_kc;
    m.ky = d.f_ky;
    m.Atau = d.f_Atau;
    m.r_out = d.f_r_out;
    m.synch = d.f_synch;
    m.spot = d.s.emitter == ODX_EMIT_SPOT;
    return m;
}

void set_launch_medium(TraceArgs &a, const DevScene &d, bool single)
{
    a.single_medium = single ? 1 : 0;
    a.med = medium_const(d);
}

bool shared_medium(const DevScene *table, int32_t n_scenes)
{
    const MedConst m0 = medium_const(table[0]);
    for (int32_t k = 1; k < n_scenes; ++k) {
        const MedConst mk = medium_const(table[k]);
        if (memcmp(&mk, &m0, sizeof(MedConst)) != 0) return false;
    }
    return true;
}

// Argument checks of odx_render for callers without a context (no message is stored).
int32_t validate_scene_table(const odx_scene *scenes, int32_t n_scenes)
{
    if (!scenes || n_scenes < 1) return ODX_ERR_INVALID_ARG;
    for (int k = 0; k < n_scenes; ++k) {
        const int32_t rc = validate_scene(nullptr, scenes[k], k, false);
        if (rc != ODX_OK) return rc;
        if (scenes[k].emitter != scenes[0].emitter || scenes[k].precision != scenes[0].precision ||
            odx::scene_planes(scenes[k]) != odx::scene_planes(scenes[0]))
            return ODX_ERR_INVALID_ARG;
    }
    return ODX_OK;
}

int32_t transfer_slots(int32_t emitter, int32_t n_freq) { return nf_slots(emitter, n_freq); }

struct CtxView {
    int device, num_sms;
    odx_launch launch;
    unsigned long long *queue;
    DevStats *stats;
};
// What the learned-surrogate code needs from a context to launch the tracer.
int32_t ctx_view(odx_ctx *ctx, CtxView *v)
{
    if (!ctx || !v) return ODX_ERR_INVALID_ARG;
    v->device = ctx->device;
    v->num_sms = ctx->num_sms;
    v->launch = ctx->launch;
    v->queue = ctx->queue;
    v->stats = ctx->stats;
    return ODX_OK;
}
}  // namespace odx

extern "C" {

const char *odx_version(void) { return kVersion; }

const char *odx_error_string(int32_t code)
{
    switch (code) {
    case ODX_OK: return "ok";
    case ODX_ERR_INVALID_ARG: return "invalid argument";
    case ODX_ERR_CUDA: return "CUDA error";
    case ODX_ERR_TIMEOUT: return "timeout";
    case ODX_ERR_DEVICE_FLAG: return "device error flag raised";
    case ODX_ERR_NO_DEVICE: return "no suitable CUDA device";
    case ODX_ERR_UNSUPPORTED: return "unsupported";
    case ODX_ERR_TOO_LARGE: return "request exceeds the fixed static scratch capacity";
    default: return "unknown error code";
    }
}

const char *odx_last_error(const odx_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int32_t odx_create(odx_ctx **out, int32_t device)
{
    if (!out) return ODX_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n)
        return ODX_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return ODX_ERR_NO_DEVICE;
    if (prop.major != 10 || prop.minor != 3) return ODX_ERR_NO_DEVICE;
    odx_ctx *ctx = new odx_ctx();
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&ctx->queue, 256) != cudaSuccess ||
        cudaMalloc(&ctx->stats, sizeof(DevStats)) != cudaSuccess ||
        cudaMemset(ctx->stats, 0, sizeof(DevStats)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->host_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        odx::prepare_fp64_kernels() != cudaSuccess) {
        odx_destroy(ctx);
        return ODX_ERR_CUDA;
    }
    *out = ctx;
    return ODX_OK;
}

int32_t odx_destroy(odx_ctx *ctx)
{
    if (!ctx) return ODX_OK;
    cudaSetDevice(ctx->device);
    if (ctx->queue) cudaFree(ctx->queue);
    if (ctx->stats) cudaFree(ctx->stats);
    if (ctx->scenes) cudaFree(ctx->scenes);
    if (ctx->hbuf) cudaFree(ctx->hbuf);
    if (ctx->flux_buf) cudaFree(ctx->flux_buf);
    if (ctx->host_stream) cudaStreamDestroy(ctx->host_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (auto &pr : ctx->events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    delete ctx;
    return ODX_OK;
}

int32_t odx_set_launch(odx_ctx *ctx, const odx_launch *L)
{
    if (!ctx || !L) return ODX_ERR_INVALID_ARG;
    if (L->block < 32 || L->block > 1024 || (L->block % 32) != 0)
        return fail(ctx, ODX_ERR_INVALID_ARG, "block must be a multiple of 32 in 32..1024");
    if (L->blocks_per_sm < 1 || L->blocks_per_sm > 64)
        return fail(ctx, ODX_ERR_INVALID_ARG, "blocks_per_sm must be 1..64");
    if (L->chunk < 0 || L->chunk > 4096)
        return fail(ctx, ODX_ERR_INVALID_ARG, "chunk must be 0 (per-path default) or 1..4096");
    if (L->persistent < 0 || L->persistent > 3)
        return fail(ctx, ODX_ERR_INVALID_ARG, "persistent must be 0, 1, 2 (auto) or 3");
    if (L->fp64_batch < 1 || L->fp64_batch > 32)
        return fail(ctx, ODX_ERR_INVALID_ARG, "fp64_batch must be 1..32");
    ctx->launch = *L;
    return ODX_OK;
}

int32_t odx_get_launch(const odx_ctx *ctx, odx_launch *L)
{
    if (!ctx || !L) return ODX_ERR_INVALID_ARG;
    *L = ctx->launch;
    return ODX_OK;
}

int32_t odx_render(odx_ctx *ctx, const odx_scene *scenes, int32_t n_scenes,
                   odx_ray_record *records, double *image, void *stream)
{
    if (!ctx) return ODX_ERR_INVALID_ARG;
    return submit(ctx, scenes, n_scenes, nullptr, -1, records, image, (cudaStream_t)stream,
                  nullptr, nullptr);
}

int32_t odx_trace_rays(odx_ctx *ctx, const odx_scene *proto, const double *rays, int64_t n,
                       odx_ray_record *records, double *image, void *stream)
{
    if (!ctx) return ODX_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, ODX_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return proto ? ODX_OK : fail(ctx, ODX_ERR_INVALID_ARG, "no prototype scene");
    return submit(ctx, proto, 1, rays, n, records, image, (cudaStream_t)stream, nullptr, nullptr);
}

int32_t odx_render_host(odx_ctx *ctx, const odx_scene *scenes, int32_t n_scenes,
                        odx_ray_record *records_host, double *image_host)
{
    if (!ctx || !scenes || n_scenes < 1 || !records_host) return ODX_ERR_INVALID_ARG;
    int64_t nr = 0, ni = 0;
    for (int k = 0; k < n_scenes; ++k) {
        if (scenes[k].n_alpha < 1 || scenes[k].n_beta < 1)
            return fail(ctx, ODX_ERR_INVALID_ARG, "scene %d: resolution must be >= 1", k);
        const int64_t p = (int64_t)scenes[k].n_alpha * scenes[k].n_beta;
        nr += p;
        ni += p * odx::scene_planes(scenes[k]);
    }
    const size_t rec_bytes = (size_t)nr * sizeof(odx_ray_record);
    const size_t img_bytes = (size_t)ni * sizeof(double);
    int32_t rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    if (ctx->hbuf_bytes < rec_bytes + img_bytes) {
        if (ctx->hbuf) ODX_CUDA(ctx, cudaFree(ctx->hbuf));
        ctx->hbuf = nullptr;
        ctx->hbuf_bytes = 0;
        ODX_CUDA(ctx, cudaMalloc(&ctx->hbuf, rec_bytes + img_bytes));
        ctx->hbuf_bytes = rec_bytes + img_bytes;
    }
    odx_ray_record *rec = (odx_ray_record *)ctx->hbuf;
    double *img = (double *)((char *)ctx->hbuf + rec_bytes);
    // A large single image is rendered in two slabs of consecutive rays, each a launch of its
    // own over the same scene table (every ray is computed exactly as in one launch): first
    // the last 7/8 of the rays, then the first 1/8, whose launch hides the device-to-host
    // copy of the larger slab (~190 GB/s pinned).  Both launches end on rows at the image's
    // edge, whose rays are short, so neither ends with a long tail of slow rays from the
    // image's centre; what stays exposed is the copy of the small slab.
    constexpr int64_t kSlabRays = int64_t(1) << 23;
    const int64_t slabs = (n_scenes == 1 && nr >= kSlabRays) ? 2 : 1;
    if (slabs == 1) {
        rc = submit(ctx, scenes, n_scenes, nullptr, -1, rec, image_host ? img : nullptr,
                    ctx->host_stream, nullptr, nullptr);
        if (rc != ODX_OK) return rc;
        ODX_CUDA(ctx, cudaMemcpyAsync(records_host, rec, rec_bytes, cudaMemcpyDeviceToHost,
                                      ctx->host_stream));
        if (image_host)
            ODX_CUDA(ctx, cudaMemcpyAsync(image_host, img, img_bytes, cudaMemcpyDeviceToHost,
                                          ctx->host_stream));
        ODX_CUDA(ctx, cudaStreamSynchronize(ctx->host_stream));
        return ODX_OK;
    }
    const int64_t planes = odx::scene_planes(scenes[0]);
    const int64_t split = nr / 8;
    const int64_t range[2][2] = {{split, nr}, {0, split}};
    cudaEvent_t done[2] = {nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess && rc == ODX_OK; ++k) {
        const int64_t b = range[k][0], end = range[k][1];
        rc = submit(ctx, scenes, 1, nullptr, -1, rec, image_host ? img : nullptr,
                    ctx->host_stream, nullptr, nullptr, b, end);
        if (rc != ODX_OK) break;
        e = cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(done[k], ctx->host_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, done[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(records_host + b, rec + b, (size_t)(end - b) * sizeof(odx_ray_record),
                                cudaMemcpyDeviceToHost, ctx->copy_stream);
        for (int64_t p = 0; p < planes && e == cudaSuccess && image_host; ++p)  // rays b .. end - 1
            e = cudaMemcpyAsync(image_host + p * nr + b, img + p * nr + b,
                                (size_t)(end - b) * sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->copy_stream);
    }
    const cudaError_t e1 = cudaStreamSynchronize(ctx->host_stream);
    const cudaError_t e2 = cudaStreamSynchronize(ctx->copy_stream);
    for (cudaEvent_t ev : done)
        if (ev) cudaEventDestroy(ev);
    if (rc != ODX_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "slab copy");
    if (e1 != cudaSuccess) return cuda_fail(ctx, e1, "render stream");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "copy stream");
    return ODX_OK;
}

int32_t odx_get_stats(odx_ctx *ctx, void *stream, odx_stats *out, int32_t reset)
{
    if (!ctx || !out) return ODX_ERR_INVALID_ARG;
    int32_t rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    DevStats d;
    cudaStream_t st = (cudaStream_t)stream;
    ODX_CUDA(ctx, cudaMemcpyAsync(&d, ctx->stats, sizeof(d), cudaMemcpyDeviceToHost, st));
    ODX_CUDA(ctx, cudaStreamSynchronize(st));
    out->rays = (int64_t)d.rays;
    out->steps_accepted = (int64_t)d.acc;
    out->steps_rejected = (int64_t)d.rej;
    out->steps_fp64 = (int64_t)d.fp64;
    out->lane_slots = (int64_t)d.slots;
    out->lane_active = (int64_t)d.active;
    out->error_flag = d.error_flag;
    out->reserved = 0;
    out->trace_launches = (int64_t)ctx->events_used;
    out->trace_ms = 0.0;
    for (size_t i = 0; i < ctx->events_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->events[i].first, ctx->events[i].second) == cudaSuccess)
            out->trace_ms += ms;
    }
    if (reset) {
        ctx->events_used = 0;
        ODX_CUDA(ctx, cudaMemsetAsync(ctx->stats, 0, sizeof(DevStats), st));
        ODX_CUDA(ctx, cudaStreamSynchronize(st));
    }
    return ODX_OK;
}

int32_t odx_set_kernel_timing(odx_ctx *ctx, int32_t on)
{
    if (!ctx) return ODX_ERR_INVALID_ARG;
    ctx->time_kernels = on != 0;
    ctx->events_used = 0;
    return ODX_OK;
}

int32_t odx_image_flux(odx_ctx *ctx, const odx_scene *scenes, int32_t n_scenes,
                       const double *image, double *flux, double *lum, void *stream)
{
    if (!ctx) return ODX_ERR_INVALID_ARG;
    if (!image || !flux) return fail(ctx, ODX_ERR_INVALID_ARG, "image and flux must be non-NULL");
    if (((uintptr_t)image & 7u) || ((uintptr_t)flux & 7u) || ((uintptr_t)lum & 7u))
        return fail(ctx, ODX_ERR_INVALID_ARG, "image, flux and lum must be 8-byte aligned");
    int32_t rc = odx::validate_scene_table(scenes, n_scenes);
    if (rc != ODX_OK) return fail(ctx, rc, "invalid scene table");
    const int32_t planes = odx::scene_planes(scenes[0]);
    for (int k = 1; k < n_scenes; ++k)
        if (scenes[k].emitter != scenes[0].emitter || odx::scene_planes(scenes[k]) != planes)
            return fail(ctx, ODX_ERR_INVALID_ARG,
                        "scene %d: all scenes of one call must share emitter and n_freq", k);
    rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    rc = ensure_scene_capacity(ctx, n_scenes);
    if (rc != ODX_OK) return rc;
    // scene table and plane table (the image layout of odx_render)
    ctx->host_scenes.resize(n_scenes);
    const size_t pr = odx::plane_ref_bytes();
    const int32_t n_planes = n_scenes * planes;
    ctx->host_planes.resize((size_t)n_planes * pr);
    int64_t ray = 0, img = 0, max_plane = 0;
    for (int k = 0; k < n_scenes; ++k) {
        const int64_t nk = (int64_t)scenes[k].n_alpha * scenes[k].n_beta;
        odx::fill_dev_scene(ctx->host_scenes[k], scenes[k], ray, nk, img);
        for (int j = 0; j < planes; ++j)
            odx::fill_plane_ref(ctx->host_planes.data() + (size_t)(k * planes + j) * pr,
                                img + (int64_t)j * nk, nk, k, j);
        max_plane = nk > max_plane ? nk : max_plane;
        ray += nk;
        img += planes * nk;
    }
    // chunks per plane from the sizes alone (the reduction tree does not depend on the GPU)
    int64_t ch = (max_plane + 4095) / 4096;
    const int32_t chunks = (int32_t)(ch < 1 ? 1 : (ch > 256 ? 256 : ch));
    const size_t need = ((ctx->host_planes.size() + 255) / 256) * 256 +
                        (size_t)n_planes * chunks * sizeof(double);
    if (need > ctx->flux_bytes) {
        if (ctx->flux_buf) cudaFree(ctx->flux_buf);
        ctx->flux_buf = nullptr;
        ctx->flux_bytes = 0;
        ODX_CUDA(ctx, cudaMalloc(&ctx->flux_buf, need));
        ctx->flux_bytes = need;
    }
    unsigned char *base = static_cast<unsigned char *>(ctx->flux_buf);
    double *partial = reinterpret_cast<double *>(base + ((ctx->host_planes.size() + 255) / 256) * 256);
    cudaStream_t st = (cudaStream_t)stream;
    ODX_CUDA(ctx, cudaMemcpyAsync(ctx->scenes, ctx->host_scenes.data(), n_scenes * sizeof(DevScene),
                                  cudaMemcpyHostToDevice, st));
    ODX_CUDA(ctx, cudaMemcpyAsync(base, ctx->host_planes.data(), ctx->host_planes.size(),
                                  cudaMemcpyHostToDevice, st));
    const cudaError_t e = odx::launch_image_flux(ctx->scenes, base, n_scenes, planes, max_plane,
                                                 image, partial, chunks, flux, lum, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "image flux launch");
    return ODX_OK;
}

int32_t odx_sync(odx_ctx *ctx, void *stream, double timeout_s)
{
    if (!ctx || !(timeout_s >= 0.0)) return ODX_ERR_INVALID_ARG;
    int32_t rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "cudaStreamQuery");
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return fail(ctx, ODX_ERR_TIMEOUT, "stream not done after %.3f s", el);
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    int32_t flag = 0;
    ODX_CUDA(ctx, cudaMemcpy(&flag, &ctx->stats->error_flag, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag) return fail(ctx, ODX_ERR_DEVICE_FLAG, "device error flag %d", flag);
    return ODX_OK;
}

double odx_torus_norm(double a, double nu, double ne_index, double T0, double T_index,
                      double r_outer)
{
    if (!isfinite(a) || fabs(a) >= 1.0 || !(nu > 0.0) || !(T0 > 0.0) || !isfinite(ne_index) ||
        !isfinite(T_index) || !isfinite(r_outer))
        return NAN;
    const double rp = 1.0 + sqrt(1.0 - a * a);
    if (!(r_outer > rp)) return NAN;
    // alpha_nu along the static equatorial path with C = 1, integrated in u = ln r with
    // 16-point Gauss-Legendre on 512 equal panels
    std::vector<double> x, w;
    gauss_legendre(16, x, w);
    const double u0 = log(rp), u1 = log(r_outer);
    const int panels = 512;
    const double du = (u1 - u0) / panels;
    double sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        const double mid = u0 + (p + 0.5) * du;
        for (int i = 0; i < 16; ++i) {
            const double r = exp(mid + 0.5 * du * x[i]);
            const double ne = exp(-ne_index * log(r));
            const double T = T0 * exp(-T_index * log(r));
            const double alpha = ne * ne / sqrt(T) * (-expm1(-nu / T)) / (2.0 * nu * nu * nu);
            sum += 0.5 * du * w[i] * alpha * r;
        }
    }
    return 1.0 / sum;
}

int32_t odx_graph_create(odx_ctx *ctx, const odx_scene *scenes, int32_t n_scenes,
                         odx_ray_record *records, double *image, odx_graph **out)
{
    if (!ctx || !out) return ODX_ERR_INVALID_ARG;
    *out = nullptr;
    if (!records || ((uintptr_t)records & 15u) != 0 || (image && ((uintptr_t)image & 7u)))
        return fail(ctx, ODX_ERR_INVALID_ARG, "records must be 16-byte aligned, image 8-byte");
    int32_t rc = odx::validate_scene_table(scenes, n_scenes);
    if (rc != ODX_OK) return fail(ctx, rc, "invalid scene table");
    rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    std::vector<DevScene> table(n_scenes);
    const int64_t nf = odx::scene_planes(scenes[0]);
    int64_t ray = 0, img = 0;
    for (int k = 0; k < n_scenes; ++k) {
        const int64_t nk = (int64_t)scenes[k].n_alpha * scenes[k].n_beta;
        odx::fill_dev_scene(table[k], scenes[k], ray, nk, img);
        ray += nk;
        img += nf * nk;
    }
    odx_graph *g = new odx_graph();
    g->ctx = ctx;
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaMalloc(&g->table, n_scenes * sizeof(DevScene));
    if (e == cudaSuccess)
        e = cudaMemcpy(g->table, table.data(), n_scenes * sizeof(DevScene), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = launch_resident(ctx, g->table, table.data(), scenes, n_scenes, ray, records, image,
                             cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        g->graph = graph;
        if (rc == ODX_OK && e2 != cudaSuccess) e = e2;
        if (rc == ODX_OK && e == cudaSuccess)
            e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    }
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess || rc != ODX_OK) {
        odx_graph_destroy(g);
        return rc != ODX_OK ? rc : cuda_fail(ctx, e, "graph capture");
    }
    *out = g;
    return ODX_OK;
}

int32_t odx_graph_launch(odx_graph *g, void *stream)
{
    if (!g || !g->exec) return ODX_ERR_INVALID_ARG;
    int32_t rc = set_device(g->ctx);
    if (rc != ODX_OK) return rc;
    ODX_CUDA(g->ctx, cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return ODX_OK;
}

int32_t odx_graph_destroy(odx_graph *g)
{
    if (!g) return ODX_OK;
    cudaSetDevice(g->ctx->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->table) cudaFree(g->table);
    delete g;
    return ODX_OK;
}

int32_t odx_autotune(odx_ctx *ctx, const odx_scene *scenes, int32_t n_scenes, void *stream,
                     odx_launch *best)
{
    if (!ctx || !best) return ODX_ERR_INVALID_ARG;
    int32_t rc = odx::validate_scene_table(scenes, n_scenes);
    if (rc != ODX_OK) return fail(ctx, rc, "invalid scene table");
    rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    int64_t nr = 0, ni = 0;
    for (int k = 0; k < n_scenes; ++k) {
        const int64_t p = (int64_t)scenes[k].n_alpha * scenes[k].n_beta;
        nr += p;
        ni += p * odx::scene_planes(scenes[k]);
    }
    const bool mixed = scenes[0].precision == ODX_MIXED;
    std::vector<odx_launch> cands;
    if (mixed) {  // warp-coherent queue, refilled lanes, one ray per thread
        for (int bps : {3, 4})
            for (int batch : {8, 16, 24}) cands.push_back({128, bps, 32, 3, batch});
        for (int bps : {3, 4})
            for (int chunk : {8, 16}) cands.push_back({128, bps, chunk, 1, 16});
        cands.push_back({128, 3, 32, 0, 16});
        cands.push_back({128, 4, 32, 0, 16});
    } else {
        for (int bps : {2, 3}) cands.push_back({128, bps, 32, 3, 16});
        for (int chunk : {16, 32}) cands.push_back({128, 2, chunk, 1, 16});
        cands.push_back({128, 2, 32, 0, 16});
    }
    void *rec = nullptr, *img = nullptr;
    ODX_CUDA(ctx, cudaMalloc(&rec, nr * sizeof(odx_ray_record)));
    cudaError_t e = cudaMalloc(&img, ni * sizeof(double));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const odx_launch saved = ctx->launch;
    odx_launch winner = saved;
    float best_ms = 1e30f;
    cudaStream_t st = (cudaStream_t)stream;
    for (size_t c = 0; c < cands.size() && e == cudaSuccess && rc == ODX_OK; ++c) {
        ctx->launch = cands[c];
        rc = submit(ctx, scenes, n_scenes, nullptr, -1, (odx_ray_record *)rec, (double *)img, st,
                    nullptr, nullptr);  // warm-up
        if (rc != ODX_OK) break;
        e = cudaEventRecord(e0, st);
        rc = submit(ctx, scenes, n_scenes, nullptr, -1, (odx_ray_record *)rec, (double *)img, st,
                    nullptr, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            winner = cands[c];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(rec);
    if (img) cudaFree(img);
    ctx->launch = (rc == ODX_OK && e == cudaSuccess) ? winner : saved;
    if (rc != ODX_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    *best = winner;
    return ODX_OK;
}

int32_t odx_fma_peak(odx_ctx *ctx, int32_t precision, double *flops)
{
    if (!ctx || !flops || (precision != ODX_FP64 && precision != ODX_MIXED))
        return ODX_ERR_INVALID_ARG;
    int32_t rc = set_device(ctx);
    if (rc != ODX_OK) return rc;
    cudaError_t e = run_fma_peak(precision, ctx->num_sms, flops);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fma peak");
    return ODX_OK;
}

}  // extern "C"
