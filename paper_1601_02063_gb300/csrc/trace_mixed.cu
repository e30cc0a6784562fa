// Mixed-precision backward ray tracer for GB300 (sm_103a).
//
// GB300 executes FP32 at 63x the FP64 rate (78.5 vs 1.25 TFLOP/s measured), and an FP64
// instruction issued by one lane of a warp costs the warp about as much as a full one.  The
// render is therefore three launches, all per-ray FP64 work done with every lane busy:
//   1. init pass (FP64, one ray per thread): initial state and constants of motion
//      (Section 2.2), horizon and ISCO radii, written into the ray's record slot as float
//      pairs (hi + lo, ~48-bit);
//   2. tracer (FP32 hot loop; persistent warps fed from the ray queue, by default 32
//      consecutive rays once all lanes of the warp are done): Cash-Karp stages in FP32; the
//      state and the transfer integrals tau, I kept as float pairs updated with error-free
//      two-sums (compensated sums); optional FP64 steps where r < r_switch, run per warp once
//      `fp64_batch` lanes need one; the final state is written back into the record slot;
//   3. finish pass (FP64, one ray per thread): null-condition and Carter-constant checks,
//      disk redshift (Eq. 2) and intensity, image in FP64, the final records.
// Per-ray arithmetic depends only on the ray's own path (the FP32/FP64 choice is made per
// lane from its own radius), so results do not depend on the launch shape.
#include "trace_mixed.cuh"

namespace odx {

// ---- pass 1: FP64 initial state, one ray per thread -------------------------------------
__global__ void __launch_bounds__(128) mixed_init_kernel(TraceArgs A)
{
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= launch_count(A)) return;
    const int64_t id = launch_first(A) + local;
    const DevScene &S = A.scenes[find_scene(A, id)];
    const ObsIn ob = ray_observer(A, S, id);
    const double a = ob.a;
    const double sgn = (S.s.convention == ODX_CONV_LITERAL) ? 1.0 : -1.0;
    const InitOut io = init_ray(ob, sgn);
    MixedInit m;
#pragma unroll
    for (int i = 0; i < 5; ++i) df_set(m.yh[i], m.yl[i], io.y[state_index(i)]);
    df_set(m.Lh, m.Ll, io.L);
    df_set(m.Qh, m.Ql, io.Q);
    const double r_isco = ray_r_isco(A, S, a);
    m.r_stop = (float)ray_r_stop(A, S, a);
    m.r_in = (float)((S.s.r_in > 0.0) ? S.s.r_in : r_isco);
    m.r_isco = (float)r_isco;
    m.a = (float)a;
    {
        const double af = (double)m.a, Ld = (double)m.Lh + (double)m.Ll;
        df_set(m.Ch, m.Cl, af * af - af * Ld);
    }
    store80(A.records + id, m);
}

// ---- pass 3: FP64 checks, redshift, intensity, final records -----------------------------
__global__ void __launch_bounds__(128) mixed_finish_kernel(TraceArgs A)
{
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= launch_count(A)) return;
    const int64_t id = launch_first(A) + local;
    const DevScene &S = A.scenes[find_scene(A, id)];
    const MixedOut o = load80<MixedOut>(A.records + id);
    const double a = A.list_mode ? A.rays[4 * id + 2] : S.s.a;
    const double L = df_get(o.Lh, o.Ll);
    double Q0 = df_get(o.Qh, o.Ql);
    double d_spot = 0.0;
    if (S.s.emitter == ODX_EMIT_SPOT) {  // the slot's Q carries the entry point's d
        d_spot = Q0;
        Q0 = init_ray(ray_observer(A, S, id), (S.s.convention == ODX_CONV_LITERAL) ? 1.0 : -1.0).Q;
    }
    double yend[6];
#pragma unroll
    for (int i = 0; i < 5; ++i) yend[state_index(i)] = df_get(o.yh[i], o.yl[i]);
    yend[3] = 0.0;
    RecordOut r;
    r.status = o.status;
    r.n_acc = o.n_acc;
    r.n_rej = o.n_rej;
    r.n_cross = o.n_cross;
    r.r_cross = (double)o.rc;
    r.phi_cross = (double)o.pc;
    const EndChecks ec = end_checks(a, L, yend);
    r.H_end = ec.H;
    r.Q_drift = (ec.Q - Q0) / fmax(fabs(Q0), 1.0);
    r.r_hit = r.phi_hit = r.g = qnan();
    r.intensity = 0.0;
    if (o.status == ODX_DISK_HIT && S.s.emitter == ODX_EMIT_SPOT) {
        r.r_hit = yend[0];
        r.phi_hit = yend[2];
        r.g = spot_redshift(S.s, yend[0], yend[1], L);
    } else if (o.status == ODX_DISK_HIT) {
        r.r_hit = yend[0];
        r.phi_hit = yend[2];
        r.g = disk_redshift(a, yend[0], L);
        const double g2 = r.g * r.g;
        r.intensity = g2 * g2 * pow(yend[0], -S.s.q_emis);
    }
    double *img = A.image ? A.image + S.img_offset + (id - S.ray_begin) : nullptr;
    if (S.s.emitter == ODX_EMIT_NT_DISK)
        r.intensity = nt_disk_planes(S, img, a, ray_r_isco(A, S, a), r.r_hit, r.g,
                                     o.status == ODX_DISK_HIT);
    if (S.s.emitter == ODX_EMIT_SPOT) {
        const double w = S.s.C_norm * exp(-d_spot * d_spot / (2.0 * S.s.spot_size * S.s.spot_size));
        r.intensity = spot_planes(S, img, w, r.g, o.status == ODX_DISK_HIT);
    }
    store_record(A.records + id, r);
    if (img && S.s.emitter != ODX_EMIT_NT_DISK && S.s.emitter != ODX_EMIT_SPOT) {
        if (S.s.emitter == ODX_EMIT_TORUS || S.s.emitter == ODX_EMIT_SYNCH) {
            const double Ij = S.s.emitter == ODX_EMIT_SYNCH ? synch_constants(S.s).Aj : 1.0;
            for (int k = 0; k < S.s.n_freq; ++k) {
                const float2 p = *reinterpret_cast<const float2 *>(img + (int64_t)k * S.n_rays);
                const double nu = S.s.freqs[k];
                img[(int64_t)k * S.n_rays] = nu * nu * nu * Ij * df_get(p.x, p.y);
            }
        } else {
            img[0] = r.intensity;
        }
    }
}

cudaError_t launch_trace_mixed(const TraceArgs &args_in, int32_t nf_slots, const odx_launch &L_in,
                               int32_t num_sms, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    TraceArgs args = args_in;
    // launch shape "auto": the warp-coherent queue (a warp takes 32 consecutive rays once all
    // its lanes are done: neighbouring pixels run the same branches together, and the queue
    // still balances the tail), 4 resident blocks per SM for launches of 2^18 rays or more
    // with up to 3 transfer slots, 3 otherwise (smaller launches, and the 8-slot kernel,
    // whose shared memory admits 3 blocks per SM)
    odx_launch L = L_in;
    if (L.persistent == 2) {
        L.persistent = 3;
        L.blocks_per_sm = (nf_slots <= 3 && args.n_total >= (1 << 18)) ? 4 : 3;
    }
    args.persistent = L.persistent;
    if (args.chunk <= 0) args.chunk = L.persistent == 3 ? 32 : 8;  // default queue chunk
    if (L.block > kMixedBlock) return cudaErrorInvalidValue;
    if (launch_count(args) <= 0) return cudaSuccess;
    const unsigned pass_blocks = (unsigned)((launch_count(args) + 127) / 128);
    mixed_init_kernel<<<pass_blocks, 128, 0, st>>>(args);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid = trace_grid(args, L, num_sms);
    if (ev0) cudaEventRecord(ev0, st);
    switch (nf_slots) {
    case 0: e = launch_mixed_nf<0>(args, L, grid, st); break;
    case 3: e = launch_mixed_nf<3>(args, L, grid, st); break;
    case 4: e = launch_mixed_nf<4>(args, L, grid, st); break;
    case 8: e = launch_mixed_nf<8>(args, L, grid, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (ev1) cudaEventRecord(ev1, st);
    mixed_finish_kernel<<<pass_blocks, 128, 0, st>>>(args);
    return cudaGetLastError();
}

}  // namespace odx
