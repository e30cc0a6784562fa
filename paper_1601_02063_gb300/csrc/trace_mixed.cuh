// Mixed-precision backward ray tracer for GB300 (sm_103a): the record slot shared by the
// three passes, and the FP32 tracing kernel with its FP32 and FP64 steps (templates).
// trace_mixed.cu holds the FP64 init and finish passes and the launch sequence;
// trace_mixed_nf{0,3,4,8}.cu instantiate the tracing kernels for 0, 3, 4 and 8 transfer
// slots, one translation unit each, so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "f32x2.cuh"
#include "kerr_device.cuh"
#include "odx_internal.h"
#include "trace_common.cuh"
#include "trace_step.cuh"

namespace odx {


// Record slot between the passes (same 80 bytes as odx_ray_record).
struct MixedInit {  // init pass -> tracer
    float yh[5], yl[5];  // r, theta, phi, p_r, p_theta (t starts at 0)
    float Lh, Ll;        // angular momentum
    float r_stop, r_in, r_isco, a;
    float Qh, Ql;        // Carter constant (Eq. 13), handed on to the finish pass
    float Ch, Cl;        // a^2 - a L (a the FP32 spin) as a pair, for the near-horizon stages
};
struct MixedOut {  // tracer -> finish pass
    int32_t status, n_acc, n_rej, n_cross;
    float rc, pc;        // first equatorial crossing r, phi (NaN if none)
    float Lh, Ll;        // angular momentum
    float yh[5], yl[5];  // final r, theta, phi, p_r, p_theta
    float Qh, Ql;        // initial Carter constant
};
static_assert(sizeof(MixedInit) == sizeof(odx_ray_record), "slot size");
static_assert(sizeof(MixedOut) == sizeof(odx_ray_record), "slot size");

// (hi, lo) += d, error-free (Knuth two-sum, then renormalisation).
__device__ __forceinline__ void df_add(float &hi, float &lo, float d)
{
    const float s = hi + d;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (d - bp);
    const float l = lo + err;
    const float t = s + l;
    lo = l - (t - s);
    hi = t;
}

__device__ __forceinline__ void df_set(float &hi, float &lo, double v)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ double df_get(float hi, float lo) { return (double)hi + (double)lo; }

template <typename T>
__device__ __forceinline__ void store80(void *dst, const T &v)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(&v);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 5; ++i) d[i] = s[i];
}

template <typename T>
__device__ __forceinline__ T load80(const void *src)
{
    T v;
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(&v);
#pragma unroll
    for (int i = 0; i < 5; ++i) d[i] = s[i];
    return v;
}

__device__ __forceinline__ int state_index(int i) { return i < 3 ? i : i + 1; }  // skip t


// ---- pass 2: FP32 tracer ------------------------------------------------------------------
constexpr int kMixedBlock = 128;  // threads per block of the tracing kernel (at most)

// Per-lane state that the FP32 stages read: registers.
template <int NF>
struct RayM {
    float yh[6];       // state high words: r, theta, phi, t, p_r, p_theta
    float th[NF + 1];  // tau high words
    float hf, hsf;     // FP32 step and error-scale step
    float Lh, af, sgnf, r_isco;
};

// Per-lane state touched once per accepted step or less: shared memory, laid out
// [field][thread] (consecutive lanes in consecutive banks), which leaves the registers to
// the stage loop.
template <int NF>
struct ColdM {
    float yl[6][kMixedBlock];  // state low words
    float tl[NF + 1][kMixedBlock];
    float Ih[NF + 1][kMixedBlock], Il[NF + 1][kMixedBlock];
    double hd[kMixedBlock], hsd[kMixedBlock];  // FP64 step and error-scale step
    float Ll[kMixedBlock], r_stop[kMixedBlock], r_start[kMixedBlock], r_in[kMixedBlock];
    float rc[kMixedBlock], pc[kMixedBlock];  // first crossing r, phi
    float Qh[kMixedBlock], Ql[kMixedBlock];  // initial Carter constant
    float Ch[kMixedBlock], Cl[kMixedBlock];  // a^2 - a L as a pair
    float hsf[kMixedBlock], r_switch[kMixedBlock];  // error-scale step, FP64 region
    int32_t mode[kMixedBlock], n_acc[kMixedBlock], n_rej[kMixedBlock], scene[kMixedBlock];
    float k1[6][kMixedBlock];                 // first stage of the current attempt
    long long id[kMixedBlock];
    int32_t n_cross[kMixedBlock], n64[kMixedBlock];
    // the Cash-Karp stage-input sums of the current attempt (acc[J]: stage J + 2), in pairs
    // of components: shared memory keeps them out of the stage loop's registers
    float2 acc[5][(NF + 5) / 2][kMixedBlock];
};

template <int NF>
__device__ __forceinline__ void write_slot(const TraceArgs &A, const DevScene &S,
                                           const RayM<NF> &R, const ColdM<NF> &C, int32_t status)
{
    const int t = threadIdx.x;
    const long long id = C.id[t];
    MixedOut o;
    o.status = status;
    o.n_acc = C.n_acc[t];
    o.n_rej = C.n_rej[t];
    o.n_cross = C.n_cross[t];
    o.rc = C.rc[t];
    o.pc = C.pc[t];
    o.Lh = R.Lh;
    o.Ll = C.Ll[t];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        o.yh[i] = R.yh[state_index(i)];
        o.yl[i] = C.yl[state_index(i)][t];
    }
    o.Qh = C.Qh[t];
    o.Ql = C.Ql[t];
    store80(A.records + id, o);
    if constexpr (NF > 0) {
        if (A.image) {
            double *img = A.image + S.img_offset + (id - S.ray_begin);
#pragma unroll
            for (int k = 0; k < NF; ++k)  // packed invariant-intensity pair, finished in pass 3
                if (k < S.s.n_freq)
                    *reinterpret_cast<float2 *>(img + (int64_t)k * S.n_rays) =
                        make_float2(C.Ih[k][t], C.Il[k][t]);
        }
    }
}

// Equatorial crossing in FP32 (the FP64 method, stopping at the FP32 resolution of
// cos(theta)); on return the crossing state y + dy is in (ch, cl) as pairs.
static __device__ __noinline__ void locate_crossing32(const Geo<float> &g, const float yh[6],
                                               const float yl[6], const float k1[6], float h,
                                               float ch[6], float cl[6])
{
    float lo = 0.f, hi = h;
    float flo = cosf(yh[1]);
    float dy[6];
    ck_geo_increment<float>(g, yh, k1, h, dy);
    const float fhi = cosf(yh[1] + dy[1]);
    float sig = lo - flo * (hi - lo) / (fhi - flo);
    if (!(sig > lo && sig < hi)) sig = 0.5f * (lo + hi);
    for (int it = 0; it < 40; ++it) {
        ck_geo_increment<float>(g, yh, k1, sig, dy);
        float yt[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) yt[i] = yh[i] + dy[i];
        float sn, F;
        sincosf(yt[1], &sn, &F);
        if (fabsf(F) <= 3e-7f) break;
        if ((F > 0.f) == (flo > 0.f)) {
            lo = sig;
            flo = F;
        } else {
            hi = sig;
        }
        float f[6];
        geodesic_rhs<float>(g, yt[0], yt[1], yt[4], yt[5], f);
        const float dF = -sn * f[1];
        float nx = sig - F / dF;
        if (!(nx > lo && nx < hi)) nx = 0.5f * (lo + hi);
        if (hi - lo <= 1e-6f * h) break;
        sig = nx;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        ch[i] = yh[i];
        cl[i] = yl[i];
        df_add(ch[i], cl[i], dy[i]);
    }
}

static __device__ __noinline__ void locate_crossing64m(const Geo<double> &g, const double y[6],
                                                const double k1[6], double h, double yc[6])
{
    double lo = 0.0, hi = h;
    double flo = cos(y[1]);
    double dy[6], y5[6];
    ck_geo_increment<double>(g, y, k1, h, dy);
    const double fhi = cos(y[1] + dy[1]);
    double sig = lo - flo * (hi - lo) / (fhi - flo);
    if (!(sig > lo && sig < hi)) sig = 0.5 * (lo + hi);
    for (int it = 0; it < 60; ++it) {
        ck_geo_increment<double>(g, y, k1, sig, dy);
#pragma unroll
        for (int i = 0; i < 6; ++i) y5[i] = y[i] + dy[i];
        double sn, F;
        sincos(y5[1], &sn, &F);
        if (fabs(F) <= 1e-14) break;
        if ((F > 0.0) == (flo > 0.0)) {
            lo = sig;
            flo = F;
        } else {
            hi = sig;
        }
        double f[6];
        geodesic_rhs<double>(g, y5[0], y5[1], y5[4], y5[5], f);
        const double dF = -sn * f[1];
        double nx = sig - F / dF;
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (hi - lo <= 1e-15 * h) break;
        sig = nx;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) yc[i] = y[i] + dy[i];
}

// FP32 torus constants of one lane's scene (Section 4.2, Eqs. 30-31), folded so that a stage
// needs one logarithm and two exponentials besides the two per frequency.  Launches whose
// rays share one medium read the same fields from the kernel parameters (MedConst).
template <int NF>
struct MediumF {
    float T_index, inv_T0, lr_pref, c2_pref, pref0;
    float nu[NF + 1], inv_nu3[NF + 1], rt_floor[NF + 1];
    float inv_kc, ky, Atau, r_out;  // synchrotron shell
    int32_t synch;
};

template <int NF>
__device__ __forceinline__ MediumF<NF> medium_f(const DevScene &S)
{
    MediumF<NF> m;
    m.T_index = S.f_T_index;
    m.inv_T0 = S.f_inv_T0;
    m.lr_pref = S.f_lr_pref;
    m.c2_pref = S.f_c2_pref;
    m.pref0 = S.f_pref0;
#pragma unroll
    for (int k = 0; k < NF + 1; ++k) {
        m.nu[k] = S.f_nu[k < ODX_MAX_FREQ ? k : 0];
        m.inv_nu3[k] = S.f_inv_nu3[k < ODX_MAX_FREQ ? k : 0];
        m.rt_floor[k] = S.f_rt_floor[k < ODX_MAX_FREQ ? k : 0];
    }
    m.inv_kc = S.f_inv_kc;
    m.ky = S.f_ky;
    m.Atau = S.f_Atau;
    m.r_out = S.f_r_out;
    m.synch = S.f_synch;
    return m;
}

// Horner evaluation of c[0] + c[1] u + ... + c[6] u^6.
__device__ __forceinline__ float poly6(const float (&c)[7], float u)
{
    float s = c[6];
#pragma unroll
    for (int i = 5; i >= 0; --i) s = fmaf(s, u, c[i]);
    return s;
}

// e^x K_2(x) in FP32 from K_2 = K_0 + (2 / x) K_1 and the polynomial approximations of
// Abramowitz & Stegun 9.8.1, 9.8.3, 9.8.5-9.8.8 (I_0, I_1 on x <= 3.75; K_0, K_1 on
// x <= 2 through ln(x / 2) I_n, and e^x sqrt(x) K_n on x >= 2).  Relative error <= 3.3e-7
// in FP32 for 1e-3 <= x <= 300 against a library K_2, the level of the trapezoidal sum
// (k2_scaled) at a fraction of its cost; the FP64 path keeps the trapezoidal sum.
__device__ __forceinline__ float k2_scaled32(float x)
{
    if (x <= 2.f) {
        constexpr float cI0[7] = {1.f, 3.5156229f, 3.0899424f, 1.2067492f, 0.2659732f,
                                  0.0360768f, 0.0045813f};
        constexpr float cI1[7] = {0.5f, 0.87890594f, 0.51498869f, 0.15084934f, 0.02658733f,
                                  0.00301532f, 0.00032411f};
        constexpr float cK0[7] = {-0.57721566f, 0.42278420f, 0.23069756f, 0.03488590f,
                                  0.00262698f, 0.00010750f, 0.00000740f};
        constexpr float cK1[7] = {1.f, 0.15443144f, -0.67278579f, -0.18156897f, -0.01919402f,
                                  -0.00110404f, -0.00004686f};
        const float t = x * (1.f / 3.75f), t2 = t * t;
        const float h = 0.5f * x, q = h * h, l = logf(h);  // accurate log: l ~ 0 near x = 2
        const float k0 = fmaf(-l, poly6(cI0, t2), poly6(cK0, q));
        const float xk1 = fmaf(x * x * l, poly6(cI1, t2), poly6(cK1, q));  // x K_1
        return __expf(x) * fmaf(2.f * xk1, __frcp_rn(x * x), k0);
    }
    constexpr float cK0[7] = {1.25331414f, -0.07832358f, 0.02189568f, -0.01062446f,
                              0.00587872f, -0.00251540f, 0.00053208f};
    constexpr float cK1[7] = {1.25331414f, 0.23498619f, -0.03655620f, 0.01504268f,
                              -0.00780353f, 0.00325614f, -0.00068245f};
    const float u = 2.f * __frcp_rn(x);
    return rsqrtf(x) * fmaf(u, poly6(cK1, u), poly6(cK0, u));
}

// FP32 transfer terms of the synchrotron shell (Eqs. 30-31 with Eqs. 37-39; the FP64 form
// is synch_rhs): nr = n_e / n_e0, iTh = 1 / Theta_e, ig = 1 / g.
template <int NF, class Med>
__device__ __forceinline__ void synch32(const Med &m, float r, float nr, float iTh, float ig,
                                        const float *tau, float *ft, float *fI)
{
    const float P = nr * ig * __frcp_rn(k2_scaled32(iTh));
    const float inu_c = m.inv_kc * iTh * iTh * sqrtf(r * __frcp_rn(nr));
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float nu0 = m.nu[k] * ig;
        const float w = __expf(__logf(nu0 * inu_c) * (-1.f / 12.f));  // x^-1/12
        const float w2 = w * w, w3 = w2 * w, w6 = w3 * w3;
        const float Mp = 4.0505f * w2 * (1.f + 0.40f * w3 + 0.5316f * w6);
        const float jt = P * Mp * __expf(iTh - 1.8899f * __frcp_rn(w2 * w2)) * __frcp_rn(nu0 * nu0);
        ft[k] = m.Atau * jt * expm1f(m.ky * nu0 * iTh);  // Eq. 30, Kirchhoff
        fI[k] = jt * __expf(-tau[k]);                     // Eq. 31
    }
}

// Hardware reciprocal (relative error ~1 ulp; the FP32 stages run at rtol ~1e-6).
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.f, x); }


// 2^a on the special-function unit (PTX ex2.approx.f32, relative error ~2^-22): with the
// identity e^y = 2^(y log2 e) the scaling of two exponents shares one packed multiply.
__device__ __forceinline__ float ex2_approx(float a)
{
    float d;
    asm("ex2.approx.f32 %0, %1;" : "=f"(d) : "f"(a));
    return d;
}
constexpr float kLog2e = 1.44269504088896341f;

// Low word of s = fl(x + y) (Knuth two-sum).
__device__ __forceinline__ float two_sum_err(float x, float y, float s)
{
    const float bp = s - x;
    return (x - (s - bp)) + (y - bp);
}

// How the stage inputs r, theta, p_r were formed: r = fl(y0r + tr) with tr = fl(h acc_r),
// and so on; with the state's low words (in shared memory) they give the stage inputs as
// pairs where the near-horizon and near-pole stages need them.
struct PairStage {
    float y0r, tr, y0t, tt, y0p, tp;
};

// sin and cos of theta = hi + lo near a pole (|sin theta| < 1/4).  There the FP32 stage
// input theta near pi carries an absolute rounding error of up to 1.2e-7, a large relative
// error in sin(theta) and in the L^2 / sin^4(theta) terms.  theta is reduced by the nearest
// multiple k pi in pair arithmetic (pi = kPiHi + kPiLo) and the reduced angle d, |d| < 0.26,
// goes through the Taylor series of sin and cos (truncation below 2e-11).
constexpr float kPiHi = 3.14159274101257324f, kPiLo = -8.74227766e-8f;
__device__ __forceinline__ void sincos_pole(float hi, float lo, float &s, float &c)
{
    const float k = rintf(hi * 0.318309886f);
    const float d = fmaf(-k, kPiHi, hi) + fmaf(-k, kPiLo, lo);
    const float d2 = d * d;
    float sd = d * (1.f - d2 * (1.f / 6.f) * (1.f - d2 * (1.f / 20.f) * (1.f - d2 * (1.f / 42.f))));
    float cd = 1.f - d2 * 0.5f * (1.f - d2 * (1.f / 12.f) * (1.f - d2 * (1.f / 30.f) *
                                                          (1.f - d2 * (1.f / 56.f))));
    if (((int)k) & 1) {
        sd = -sd;
        cd = -cd;
    }
    s = sd;
    c = cd;
}

// Near the horizon (Delta < r^2 / 4) F = 2 Sigma H is the difference of two terms of size
// P^2 / Delta that cancel to the size of the constraint violation, and Delta itself loses
// its leading digits.  With FP32 stage inputs the rounding of r alone makes F, and through
// it dp_theta/ds, noise of order one there, which stalls the step control of rays with small
// p_theta.  In that region Delta, Delta p_r - P and so F are formed in float-pair arithmetic
// from the stage inputs' low words.
template <class Cold>
__device__ __forceinline__ void near_horizon(float r, float pr, float a, const PairStage &ps,
                                             const Cold &C, float &Del, float &D, float &S)
{
    const int t = threadIdx.x;
    const float rl = two_sum_err(ps.y0r, ps.tr, r) + C.yl[0][t];
    const float pl = two_sum_err(ps.y0p, ps.tp, pr) + C.yl[4][t];
    const float Ch = C.Ch[t], Cl = C.Cl[t];
    const float q2 = __fmul_rn(r, r);  // r^2 = q2 + q2e (products kept out of contractions)
    const float q2e = fmaf(2.f * r, rl, fmaf(r, r, -q2));
    const float a2h = __fmul_rn(a, a), a2l = fmaf(a, a, -a2h);
    // Delta = r^2 - 2 r + a^2 (q2 - 2 r is exact for 1 <= r <= 4, Sterbenz)
    const float d1 = q2 - 2.f * r;
    float Dh = d1 + a2h;
    float Dl = two_sum_err(d1, a2h, Dh) + q2e - 2.f * rl + a2l;
    const float Ds = Dh + Dl;
    Dl = Dl - (Ds - Dh);
    Dh = Ds;
    // u = Delta p_r, P = r^2 + (a^2 - a L), D = u - P
    const float uh = __fmul_rn(Dh, pr);
    const float ul = fmaf(Dl, pr, fmaf(Dh, pl, fmaf(Dh, pr, -uh)));
    const float Ph = q2 + Ch;
    const float Pl = two_sum_err(q2, Ch, Ph) + q2e + Cl;
    const float dh = uh - Ph;
    D = dh + (two_sum_err(uh, -Ph, dh) + (ul - Pl));
    S = uh + Ph;
    Del = Dh;
}

// FP32 right-hand side of one stage: geodesic (Eqs. 4, 5, 9, 12, 14, 15, with the
// super-Hamiltonian terms F of the FP64 form) and, for NF > 0, the torus transfer terms
// (Eq. 2 redshift, Eqs. 30-31).  in = (r, theta, p_r, p_theta, tau_1..tau_NF).
// Frequency slots past the scene's n_freq repeat its last frequency (never written out).
// MK, the medium kind of the launch: 0 read per lane from the medium (batched scenes),
// 1 the torus (or no medium), 2 the synchrotron shell, 3 the hot spot (no medium; its step
// control and entry test compiled in): single-medium launches carry no other emitter's code.
template <int NF, int MK, class Med, class Cold>
__device__ __forceinline__ void derivs32(const Geo<float> &g, const Med &m, float r_isco,
                                         const float *in, const PairStage &ps, const Cold &C,
                                         float f[6], float *ft, float *fI)
{
    const float r = in[0], pr = in[2], pth = in[3];
    float s, c;
    __sincosf(in[1], &s, &c);  // |x| <= pi up to pole passages: abs. error <= 2^-21.4
    if (fabsf(s) < 0.25f)
        sincos_pole(in[1], two_sum_err(ps.y0t, ps.tt, in[1]) + C.yl[1][threadIdx.x], s, c);
    s = fmaxf(s, 1e-8f);
    const float a = g.a, L = g.L;
    const float r2 = r * r, a2 = a * a, s2 = s * s;
    const float Sig = r2 + a2 * c * c;
    float Del = r2 - 2.f * r + a2;
    const bool nh = Del < 0.25f * r2;
    float Dm = 0.f, Sm = 0.f;  // Delta p_r -+ P (near the horizon)
    if (nh) near_horizon(r, pr, a, ps, C, Del, Dm, Sm);
    const float iSD = rcp_fast(Sig * Del);
    const float iS = Del * iSD;
    const float iD = Sig * iSD;
    const float is = rcp_fast(s);
    const float is2 = is * is;
    const float rr = r2 + a2;
    const float P = rr - a * L;
    const float q = L * is - a * s;
    const float pr2 = pr * pr, pth2 = pth * pth;
    const float F = nh ? fmaf(Dm * Sm, iD, pth2 + q * q) : Del * pr2 + pth2 + q * q - P * P * iD;
    const float kap = pth2 + L * L * is2 + a2 * s2;
    const float rm1 = r - 1.f;
    const float twor = 2.f * r;
    // the direction sign sgn is carried by the geodesic step size (h_geo = sgn h)
    f[0] = Del * pr * iS;
    f[1] = pth * iS;
    f[2] = (twor * a + (Sig - twor) * L * is2) * iSD;
    f[3] = 1.f + (twor * rr - twor * a * L) * iSD;
    f[4] = (-kap * rm1 + twor * rr - 2.f * a * L) * iSD - 2.f * pr2 * rm1 * iS +
           F * (rm1 * iSD + r * iS * iS);
    f[5] = s * c * iS * (L * L * is2 * is2 - a2) - a2 * s * c * F * iS * iS;
    if constexpr (NF > 0) {
        if (r < C.r_stop[threadIdx.x]) {  // the medium ends at the stopping radius
#pragma unroll
            for (int k = 0; k < NF; ++k) ft[k] = fI[k] = 0.f;
            return;
        }
        // Keplerian flow where r >= r_ISCO and timelike, else ZAMO; 1/g = u^t (1 - Omega L)
        const float A = rr * rr - a2 * Del * s2;
        const float gtt = -(1.f - twor * iS);
        const float gtp = -twor * a * s2 * iS;
        const float gpp = A * s2 * iS;
        float Om = rcp_fast(r * r * rsqrtf(r) + a);
        float N = gtt + 2.f * gtp * Om + gpp * Om * Om;
        if (!(r >= r_isco && N < 0.f)) {  // ZAMO: g_tt - g_tphi^2 / g_phiphi = -Sigma Delta / A
            const float iA = rcp_fast(A);
            Om = twor * a * iA;
            N = -Sig * Del * iA;
        }
        const float ig = (1.f - Om * L) * rsqrtf(-N);
        const float lr = __logf(r);
        const bool synch = MK == 2 || (MK == 0 && m.synch != 0);
        if (synch) {
            if (r <= m.r_out) {
                const float nr = __expf(m.lr_pref * lr + m.c2_pref * c * c);
                synch32<NF>(m, r, nr, m.inv_T0 * __expf(m.T_index * lr), ig, in + 4, ft, fI);
            } else {
#pragma unroll
                for (int k = 0; k < NF; ++k) ft[k] = fI[k] = 0.f;
            }
            return;
        }
        const float gg = rcp_fast(ig);
        // C n_e^2 T_e^-1/2 g^2, and nu0 / T_e per unit observed frequency
        const float Q = m.pref0 * __expf(m.lr_pref * lr + m.c2_pref * c * c) * gg * gg;
        const float xi = ig * m.inv_T0 * __expf(m.T_index * lr);
        // two frequencies at a time (slot NF of the arrays is padding when NF is odd)
#pragma unroll
        for (int k = 0; k < NF; k += 2) {
            const float2 x = mul2(make_float2(m.nu[k], m.nu[k + 1]), dup2(xi));
            // C n_e^2 T_e^-1/2 / (g nu0^3)
            const float2 w = mul2(make_float2(m.inv_nu3[k], m.inv_nu3[k + 1]), dup2(Q));
            const float2 tau = make_float2(in[4 + k], k + 1 < NF ? in[5 + k] : 0.f);
            // exponents in base 2: -x log2(e) and -(x + tau) log2(e)
            const float2 ax = mul2(x, dup2(-kLog2e)), at = fma2(tau, dup2(-kLog2e), ax);
            const float2 em = make_float2(ex2_approx(ax.x), ex2_approx(ax.y));  // e^-x
            // (1 - e^-x) / 2: directly for x > 1/32, else x (1/2 - x (1/4 - x / 12)) (the
            // subtraction would lose up to 5 bits there); the halving is exact either way
            const float2 big = fma2(em, dup2(-0.5f), dup2(0.5f));
            const float2 ser =
                mul2(x, fma2(x, fma2(x, dup2(1.f / 12.f), dup2(-0.25f)), dup2(0.5f)));
            const float2 om = make_float2(x.x > 0.03125f ? big.x : ser.x,
                                          x.y > 0.03125f ? big.y : ser.y);
            const float2 ftk = mul2(w, om);                                          // Eq. 30
            const float2 fIk = mul2(w, make_float2(ex2_approx(at.x), ex2_approx(at.y)));  // Eq. 31
            ft[k] = ftk.x;
            fI[k] = fIk.x;
            if (k + 1 < NF) {
                ft[k + 1] = ftk.y;
                fI[k + 1] = fIk.y;
            }
        }
    }
}

// Sign of cos(theta) for theta = hi + lo: the hardware cosine away from the zeros, the
// accurate one corrected by the low word near them.
__device__ __forceinline__ bool cos_positive(float hi, float lo)
{
    const float c = __cosf(hi);
    if (fabsf(c) > 1e-3f) return c > 0.f;
    float sn, cs;
    sincosf(hi, &sn, &cs);
    return cs - lo * sn > 0.f;
}

// Record the crossing; returns true when the ray stops on the thin disk (the crossing state
// becomes the final state).
template <int NF>
__device__ __forceinline__ bool on_crossing(const DevScene &S, RayM<NF> &R, ColdM<NF> &C,
                                            const float ch[6], const float cl[6])
{
    const int t = threadIdx.x;
    const int n = ++C.n_cross[t];
    if (n == 1) {
        C.rc[t] = ch[0];
        C.pc[t] = ch[2];
    }
    if (disk_emitter(S.s.emitter) && ch[0] >= C.r_in[t] && ch[0] <= S.f_r_out) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            R.yh[i] = ch[i];
            C.yl[i][t] = cl[i];
        }
        return true;
    }
    return false;
}

// FP32 distance from the hot spot's sphere d = 4 r_spot (the spot test itself and the entry
// point run in FP64): the centre's azimuth at the emission time t_obs - sgn t.
__device__ __forceinline__ float spot_gap32(const DevScene &S, float r, float th, float ph,
                                            float t, float sgn, float a)
{
    float sp, cp, ss, cs;
    sincosf(ph, &sp, &cp);
    sincosf(S.f_spot_ph - S.f_spot_om * sgn * t, &ss, &cs);
    const float R = sqrtf(r * r + a * a), z = r * cosf(th);
    const float dx = R * cp - S.f_spot_Rs * cs, dy = R * sp - S.f_spot_Rs * ss;
    return sqrtf(dx * dx + dy * dy + z * z) - S.f_spot_R4;
}

// Attempts after which a ray leaves the FP32 stages for good (typical rays take 100-400).
constexpr int kFp32Stall = 4096;

// One FP32 Cash-Karp attempt.  Returns the new status.
//
// The six stages run as a loop around one inlined right-hand side (one copy of its code in
// the instruction cache, no call).  Each stage's derivative is folded at once into the
// inputs of the later stages (acc[j]: the weighted sum for stage j + 1), the fifth-order
// sum and the error estimate, so no stage derivative is kept; t and phi, which no
// right-hand side reads, enter only those two sums.  The first stage is evaluated afresh
// at every attempt (a rejected attempt repeats it exactly).
template <int NF, int MK, class Med>
__device__ __forceinline__ int32_t step32(const DevScene &S, RayM<NF> &R, ColdM<NF> &C,
                                          const Med &mf)
{
    const int t = threadIdx.x;
    constexpr int NG = 4 + NF;  // stage inputs: r, theta, p_r, p_theta, tau_k
    const Geo<float> g{R.af, R.Lh, R.sgnf};
    if (C.mode[t] != 0) {  // (re)enter FP32
        if (C.mode[t] == 1) R.hf = (float)C.hd[t];
        C.hsf[t] = R.hf;
        C.mode[t] = 0;
    }
    const float h = R.hf;
    const float hg = R.sgnf * h;  // geodesic components: dy/ds = sgn f
    // stage inputs in pairs: (r, theta), (p_r, p_theta), (tau_0, tau_1), ... (the last pair's
    // second slot is padding when NF is odd); the stage sums below use packed FMAs
    constexpr int NP = (NG + 1) / 2;
    float2 y0[NP];
    y0[0] = make_float2(R.yh[0], R.yh[1]);
    y0[1] = make_float2(R.yh[4], R.yh[5]);
#pragma unroll
    for (int q = 2; q < NP; ++q) y0[q] = make_float2(R.th[2 * q - 4], R.th[2 * q - 3]);
    float in[NG + 1];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        in[2 * q] = y0[q].x;
        in[2 * q + 1] = y0[q].y;
    }
    PairStage ps{y0[0].x, 0.f, y0[0].y, 0.f, y0[1].x, 0.f};
    // acc[J]: weighted slope sums for the input of stage J + 1; de[i] = (dy_i, e_i): fifth-
    // order sum and error estimate of geodesic component i; dIe[k] = (dI_k, eI_k) of the
    // intensities; dt[q]: fifth-order sums of tau_2q, tau_2q+1
    static_assert((NF + 5) / 2 == NP, "pairs of stage inputs");
    float2 de[6], dIe[NF + 1], dt[NP];
    auto acc = C.acc;  // [J][pair][thread]

#define ODX_ACC(J, COEF)                                                   \
    _Pragma("unroll") for (int q = 0; q < NP; ++q) acc[J][q][t] = fma2(dup2((float)(COEF)), kf[q], acc[J][q][t]);
#define ODX_NEXT(J)                                                        \
    {                                                                      \
        const float2 a0 = acc[J][0][t], a1 = acc[J][1][t];                 \
        const float2 tg = mul2(dup2(hg), a0);                              \
        ps.tr = tg.x;                                                      \
        ps.tt = tg.y;                                                      \
        ps.tp = __fmul_rn(hg, a1.x);                                       \
        const float2 rt = add2(y0[0], tg);                                 \
        in[0] = rt.x;                                                      \
        in[1] = rt.y;                                                      \
        in[2] = __fadd_rn(y0[1].x, ps.tp);                                 \
        in[3] = fmaf(hg, a1.y, y0[1].y);                                   \
        _Pragma("unroll") for (int q = 2; q < NP; ++q) {                   \
            const float2 v = fma2(dup2(h), acc[J][q][t], y0[q]);           \
            in[2 * q] = v.x;                                               \
            in[2 * q + 1] = v.y;                                           \
        }                                                                  \
    }
#define ODX_SUMS(B, E)                                                     \
    _Pragma("unroll") for (int i = 0; i < 6; ++i)                          \
        de[i] = fma2(make_float2((float)(B), (float)(E)), dup2(f[i]), de[i]); \
    _Pragma("unroll") for (int k = 0; k < NF; ++k)                         \
        dIe[k] = fma2(make_float2((float)(B), (float)(E)), dup2(fI[k]), dIe[k]); \
    _Pragma("unroll") for (int q = 2; q < NP; ++q) dt[q] = fma2(dup2((float)(B)), kf[q], dt[q]);

#pragma unroll 1
    for (int st = 0; st < 6; ++st) {
        float f[6], ft[NF + 1], fI[NF + 1];
        derivs32<NF, MK>(g, mf, R.r_isco, in, ps, C, f, ft, fI);
        float2 kf[NP];
        kf[0] = make_float2(f[0], f[1]);
        kf[1] = make_float2(f[4], f[5]);
#pragma unroll
        for (int q = 2; q < NP; ++q) kf[q] = make_float2(ft[2 * q - 4], ft[2 * q - 3]);
        switch (st) {
        case 0:
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                acc[0][q][t] = mul2(dup2((float)CK_A21), kf[q]);
                acc[1][q][t] = mul2(dup2((float)CK_A31), kf[q]);
                acc[2][q][t] = mul2(dup2((float)CK_A41), kf[q]);
                acc[3][q][t] = mul2(dup2((float)CK_A51), kf[q]);
                acc[4][q][t] = mul2(dup2((float)CK_A61), kf[q]);
                dt[q] = mul2(dup2((float)CK_B1), kf[q]);
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                C.k1[i][t] = R.sgnf * f[i];
                de[i] = mul2(make_float2((float)CK_B1, (float)CK_E1), dup2(f[i]));
            }
#pragma unroll
            for (int k = 0; k < NF; ++k)
                dIe[k] = mul2(make_float2((float)CK_B1, (float)CK_E1), dup2(fI[k]));
            ODX_NEXT(0)
            break;
        case 1:  // b2 = e2 = 0
            ODX_ACC(1, CK_A32)
            ODX_ACC(2, CK_A42)
            ODX_ACC(3, CK_A52)
            ODX_ACC(4, CK_A62)
            ODX_NEXT(1)
            break;
        case 2:
            ODX_ACC(2, CK_A43)
            ODX_ACC(3, CK_A53)
            ODX_ACC(4, CK_A63)
            ODX_SUMS(CK_B3, CK_E3)
            ODX_NEXT(2)
            break;
        case 3:
            ODX_ACC(3, CK_A54)
            ODX_ACC(4, CK_A64)
            ODX_SUMS(CK_B4, CK_E4)
            ODX_NEXT(3)
            break;
        case 4:  // b5 = 0
            ODX_ACC(4, CK_A65)
#pragma unroll
            for (int i = 0; i < 6; ++i) de[i].y = fmaf((float)CK_E5, f[i], de[i].y);
#pragma unroll
            for (int k = 0; k < NF; ++k) dIe[k].y = fmaf((float)CK_E5, fI[k], dIe[k].y);
            ODX_NEXT(4)
            break;
        default:
            ODX_SUMS(CK_B6, CK_E6)
            break;
        }
    }
#undef ODX_ACC
#undef ODX_NEXT
#undef ODX_SUMS
    float dy[6], e[6], dtau[NF + 1], dI[NF + 1], eI[NF + 1];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        dy[i] = de[i].x;
        e[i] = de[i].y;
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        dI[k] = dIe[k].x;
        eI[k] = dIe[k].y;
        dtau[k] = (k & 1) ? dt[2 + k / 2].y : dt[2 + k / 2].x;
    }

    float errmax = 0.f;
    bool nan_err = false;  // fmaxf drops a NaN operand: track it, it rejects the step
    const float hs = C.hsf[t];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float sc = fabsf(R.yh[i]) + fabsf(hs * C.k1[i][t]) + 1e-30f;
        const float v = __fdividef(fabsf(hg * e[i]), sc);
        nan_err |= isnan(v);
        errmax = fmaxf(errmax, v);
    }
    // the intensities under the step control, scaled by |I| + |h dI/ds| (this step's slope)
    // + the floor (ODX_RT_RIDE: infinite floors)
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const float sc = fabsf(C.Ih[k][t]) + fabsf(h * dI[k]) + mf.rt_floor[k];
        const float v = __fdividef(fabsf(h * eI[k]), sc);
        nan_err |= isnan(v);
        errmax = fmaxf(errmax, v);
    }
    errmax = __fdividef(errmax, S.f_rtol32);
    if (nan_err || isnan(errmax)) {  // reject; the ray goes on in FP64 steps
        errmax = INFINITY;
        C.r_switch[t] = INFINITY;
    }
    if (!(errmax <= 1.f)) {
        ++C.n_rej[t];
        R.hf = fmaxf(0.9f * h * __powf(errmax, -0.25f), 0.1f * h);
        // a step that collapses below 1e-6 r (rays passing a pole when the observer sits on
        // the axis) is beyond the FP32 stages: FP64 steps for the rest of the ray
        if (R.hf < 1e-6f * R.yh[0]) C.r_switch[t] = INFINITY;
        return R.hf < 1e-12f ? ODX_NUMERR : ODX_RUNNING;
    }
    ++C.n_acc[t];
    // a ray still in the FP32 stages after kFp32Stall attempts (rays passing a pole when the
    // observer sits on the axis can creep on at a noise-limited step) finishes in FP64 steps
    if (C.n_acc[t] + C.n_rej[t] > kFp32Stall) C.r_switch[t] = INFINITY;
    const float h_next = (errmax > 1.89e-4f) ? 0.9f * h * __powf(errmax, -0.2f) : 5.f * h;
#pragma unroll
    for (int i = 0; i < 6; ++i) dy[i] = __fmul_rn(dy[i], hg);  // rounded before the two-sums
    {
        float nh = R.yh[1], nl = C.yl[1][t];
        const bool c0 = cos_positive(nh, nl);
        df_add(nh, nl, dy[1]);
        if (c0 != cos_positive(nh, nl)) {
            float yl[6], k1[6], ch[6], cl[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                yl[i] = C.yl[i][t];
                k1[i] = C.k1[i][t];
            }
            locate_crossing32(g, R.yh, yl, k1, h, ch, cl);
            if (on_crossing<NF>(S, R, C, ch, cl)) return ODX_DISK_HIT;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float lo = C.yl[i][t];
        df_add(R.yh[i], lo, dy[i]);
        C.yl[i][t] = lo;
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        float tlo = C.tl[k][t], ih = C.Ih[k][t], il = C.Il[k][t];
        df_add(R.th[k], tlo, __fmul_rn(h, dtau[k]));
        df_add(ih, il, __fmul_rn(h, dI[k]));
        C.tl[k][t] = tlo;
        C.Ih[k][t] = ih;
        C.Il[k][t] = il;
    }
    if (R.yh[0] < C.r_stop[t]) return ODX_CAPTURED;
    // escape: dr/ds = sgn Delta p_r / Sigma has the sign of sgn p_r outside the horizon
    if (R.sgnf * R.yh[4] > 0.f && R.yh[0] > C.r_start[t]) return ODX_ESCAPED;
    R.hf = fminf(h_next, S.f_hmax_frac * R.yh[0]);
    if constexpr (MK == 3) {  // steps near the spot, FP64 within r_spot / 2
        const float gap = spot_gap32(S, R.yh[0], R.yh[1], R.yh[2], R.yh[3] + C.yl[3][t], R.sgnf,
                                     R.af);
        const float sz = 0.25f * S.f_spot_R4;
        R.hf = fminf(R.hf, fmaxf(0.5f * gap, 0.25f * sz));
        if (gap < 0.5f * sz) C.r_switch[t] = INFINITY;
    }
    C.hsf[t] = R.hf;
    return ODX_RUNNING;
}

// One FP64 Cash-Karp attempt on the pair state (FP64 tolerance rtol).  The first stage is
// evaluated afresh in FP64: FP64 steps are rare and batched, and keeping an FP64 first stage
// alive across the FP32 steps would cost 2 x (6 + 2 NF) registers on every step.
template <int NF, int MK>
__device__ __noinline__ int32_t step64(const TraceArgs &A, const DevScene &S, RayM<NF> &R,
                                       ColdM<NF> &C, float r_isco)
{
    const int t = threadIdx.x;
    const double a = A.list_mode ? A.rays[4 * C.id[t] + 2] : S.s.a;
    const double L = df_get(R.Lh, C.Ll[t]);
    const Geo<double> g{a, L, (double)R.sgnf};
    MediumT<double> md{};
    if constexpr (NF > 0) {
        load_medium_t<double>(S, (double)r_isco, (double)C.r_stop[t], md);
        // a single-medium launch compiles only its own emitter into the FP64 stages
        if constexpr (MK == 1) md.synch = 0;
        if constexpr (MK == 2) md.synch = 1;
    }
    double y[6], tau[NF + 1], k1[6], kt1[NF + 1], kI1[NF + 1];
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = df_get(R.yh[i], C.yl[i][t]);
#pragma unroll
    for (int k = 0; k < NF; ++k) tau[k] = df_get(R.th[k], C.tl[k][t]);
    derivs<double, NF>(g, md, y, tau, k1, kt1, kI1);
    if (C.mode[t] != 1) {  // entering FP64
        C.hd[t] = (double)R.hf;
        C.hsd[t] = C.hd[t];
        C.mode[t] = 1;
    }
    ++C.n64[t];
    const double h = C.hd[t];
    double dy[6], e[6], dtau[NF + 1], dI[NF + 1], eI[NF + 1];
    ck_attempt<double, NF>(g, md, y, k1, tau, kt1, kI1, h, dy, e, dtau, dI, eI);
    double errmax = 0.0;
    bool nan_err = false;  // fmax drops a NaN operand: track it, it rejects the step
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double sc = fabs(y[i]) + fabs(C.hsd[t] * k1[i]) + 1e-30;
        const double v = fabs(e[i] / sc);
        nan_err |= isnan(v);
        errmax = fmax(errmax, v);
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const double sc = fabs(df_get(C.Ih[k][t], C.Il[k][t])) + fabs(C.hsd[t] * kI1[k]) +
                          md.I_floor[k];
        const double v = fabs(eI[k] / sc);
        nan_err |= isnan(v);
        errmax = fmax(errmax, v);
    }
    errmax /= S.s.rtol;
    if (nan_err || isnan(errmax)) errmax = INFINITY;
    if (!(errmax <= 1.0)) {
        ++C.n_rej[t];
        C.hd[t] = fmax(0.9 * h * pow(errmax, -0.25), 0.1 * h);
        return C.hd[t] < 1e-12 ? ODX_NUMERR : ODX_RUNNING;
    }
    ++C.n_acc[t];
    const double h_next = (errmax > 1.89e-4) ? 0.9 * h * pow(errmax, -0.2) : 5.0 * h;
    if ((cos(y[1]) > 0.0) != (cos(y[1] + dy[1]) > 0.0)) {
        double yc[6];
        locate_crossing64m(g, y, k1, h, yc);
        float ch[6], cl[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) df_set(ch[i], cl[i], yc[i]);
        if (on_crossing<NF>(S, R, C, ch, cl)) return ODX_DISK_HIT;
    }
    double spot_d = 0.0;  // distance from the spot's centre at the step's end
    if constexpr (MK == 3) {  // first entry into the hot spot
        double y5[6], d;
#pragma unroll
        for (int i = 0; i < 6; ++i) y5[i] = y[i] + dy[i];
        const double q5 = spot_region(S.s, g.sgn, y5, spot_d);
        if (q5 < 0.0) {
            double yc[6];
            // the entry point to 4e-9 r_spot (the FP64 path bisects to 2^-60 of the step;
            // both are far inside the reduced-precision intensity bar)
            enter_spot64(g, S.s, y, k1, h, q5, 4e-9 * S.s.spot_size, yc);
            spot_region(S.s, g.sgn, yc, d);
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                float lo;
                df_set(R.yh[i], lo, yc[i]);
                C.yl[i][t] = lo;
            }
            df_set(C.Qh[t], C.Ql[t], d);  // the record slot's Q carries d to the finish pass
            return ODX_DISK_HIT;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        y[i] += dy[i];
        float lo;
        df_set(R.yh[i], lo, y[i]);
        C.yl[i][t] = lo;
    }
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        tau[k] += dtau[k];
        float tlo, ih, il;
        df_set(R.th[k], tlo, tau[k]);
        df_set(ih, il, df_get(C.Ih[k][t], C.Il[k][t]) + dI[k]);
        C.tl[k][t] = tlo;
        C.Ih[k][t] = ih;
        C.Il[k][t] = il;
    }
    if (R.yh[0] < C.r_stop[t]) return ODX_CAPTURED;
    // escape test: dr/ds = sgn Delta p_r / Sigma has the sign of sgn p_r outside the horizon
    if (R.sgnf * R.yh[4] > 0.f && R.yh[0] > C.r_start[t]) return ODX_ESCAPED;
    C.hd[t] = fmin(h_next, S.s.hmax_frac * y[0]);
    if constexpr (MK == 3) {  // back to FP32 once clear of the spot (y is y5)
        C.hd[t] = fmin(C.hd[t], spot_cap(S.s, spot_d));
        if (spot_d - 4.0 * S.s.spot_size > S.s.spot_size) C.r_switch[t] = (float)S.s.r_switch;
    }
    C.hsd[t] = C.hd[t];
    R.hf = (float)C.hd[t];
    return ODX_RUNNING;
}

// MINB: resident 128-thread blocks per SM the register allocation is capped for.
// SINGLE: every ray shares the launch's medium (A.med, read from the kernel parameters, no
// registers); otherwise each lane keeps its scene's constants.
template <int NF, int MINB, bool SINGLE, int MK>
__global__ void __launch_bounds__(kMixedBlock, MINB)
    trace_mixed_kernel(const __grid_constant__ TraceArgs A)
{
    __shared__ ColdM<NF> C;
    // per-warp counters: slots/active written by lane 0 only, the rest by finishing lanes
    __shared__ unsigned long long wstat[kMixedBlock / 32][6];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (lane < 6) wstat[warp][lane] = 0ull;
    __syncwarp();
    RayM<NF> R;
    MediumF<NF> mf{};
    bool live = false;
    WarpQueue q;
    q.init(A);

    for (;;) {
        int64_t id;
        q.refill(A, lane, live, id);
        if (id >= 0) {  // refill from the init pass's slot: no FP64 work here
            const int32_t sidx = find_scene(A, id);
            const DevScene &S = A.scenes[sidx];
            const MixedInit m = load80<MixedInit>(A.records + id);
            C.id[t] = id;
            C.scene[t] = sidx;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                R.yh[state_index(i)] = m.yh[i];
                C.yl[state_index(i)][t] = m.yl[i];
            }
            R.yh[3] = 0.f;
            C.yl[3][t] = 0.f;
            R.Lh = m.Lh;
            C.Ll[t] = m.Ll;
            R.af = m.a;
            R.sgnf = (S.s.convention == ODX_CONV_LITERAL) ? 1.f : -1.f;
            C.r_switch[t] = (float)S.s.r_switch;
            C.r_stop[t] = m.r_stop;
            C.r_in[t] = m.r_in;
            C.r_start[t] = m.yh[0];
            C.Ch[t] = m.Ch;
            C.Cl[t] = m.Cl;
#pragma unroll
            for (int k = 0; k < NF + 1; ++k) {
                R.th[k] = 0.f;
                C.tl[k][t] = C.Ih[k][t] = C.Il[k][t] = 0.f;
            }
            C.rc[t] = C.pc[t] = __int_as_float(0x7fc00000);
            C.Qh[t] = m.Qh;
            C.Ql[t] = m.Ql;
            C.n_acc[t] = C.n_rej[t] = 0;
            C.n_cross[t] = C.n64[t] = 0;
            R.hf = fminf((float)S.s.h0, S.f_hmax_frac * m.yh[0]);
            C.hsf[t] = R.hf;
            C.mode[t] = -1;
            R.r_isco = m.r_isco;
            if constexpr (!SINGLE) mf = medium_f<NF>(S);
            live = true;
        }
        const unsigned act = __ballot_sync(kFull, live);
        if (act == 0u) break;
        if (lane == 0) {
            wstat[warp][4] += 32;
            wstat[warp][5] += __popc(act);
        }
        // per-lane precision of this step, from the lane's own radius
        const bool want64 = live && (R.yh[0] < C.r_switch[t]);
        const unsigned b64 = __ballot_sync(kFull, want64);
        const unsigned b32 = act & ~b64;
        const bool run64 = b64 != 0u && (__popc(b64) >= A.fp64_batch || b32 == 0u);
        const bool mine = run64 ? want64 : (live && !want64);
        if (mine) {
            const DevScene &S = A.scenes[A.n_scenes == 1 ? 0 : C.scene[t]];
            int32_t status;
            if (run64) {
                // the FP64 step works on a copy: only this rare path pays for moving the
                // register state through local memory
                RayM<NF> r64 = R;
                status = step64<NF, MK>(A, S, r64, C, R.r_isco);
                R = r64;
            } else {
                if constexpr (SINGLE)
                    status = step32<NF, MK>(S, R, C, A.med);
                else
                    status = step32<NF, MK>(S, R, C, mf);
            }
            if (status == ODX_RUNNING && C.n_acc[t] + C.n_rej[t] >= S.s.max_steps)
                status = ODX_MAXSTEPS;
            if (status != ODX_RUNNING) {
                write_slot<NF>(A, S, R, C, status);
                atomicAdd(&wstat[warp][0], 1ull);
                atomicAdd(&wstat[warp][1], (unsigned long long)C.n_acc[t]);
                atomicAdd(&wstat[warp][2], (unsigned long long)C.n_rej[t]);
                atomicAdd(&wstat[warp][3], (unsigned long long)C.n64[t]);
                live = false;
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        atomicAdd(&A.stats->rays, wstat[warp][0]);
        atomicAdd(&A.stats->acc, wstat[warp][1]);
        atomicAdd(&A.stats->rej, wstat[warp][2]);
        atomicAdd(&A.stats->fp64, wstat[warp][3]);
        atomicAdd(&A.stats->slots, wstat[warp][4]);
        atomicAdd(&A.stats->active, wstat[warp][5]);
    }
}

template <int NF, bool SINGLE, int MK>
cudaError_t launch_mixed_nf(const TraceArgs &args, const odx_launch &L, dim3 grid, cudaStream_t st)
{
    const dim3 block(L.block);
    switch (L.blocks_per_sm <= 2 ? 2 : (L.blocks_per_sm >= 4 ? 4 : 3)) {
    case 2: trace_mixed_kernel<NF, 2, SINGLE, MK><<<grid, block, 0, st>>>(args); break;
    case 3: trace_mixed_kernel<NF, 3, SINGLE, MK><<<grid, block, 0, st>>>(args); break;
    default: trace_mixed_kernel<NF, 4, SINGLE, MK><<<grid, block, 0, st>>>(args); break;
    }
    return cudaGetLastError();
}

template <int NF>
cudaError_t launch_mixed_nf(const TraceArgs &args, const odx_launch &L, dim3 grid, cudaStream_t st)
{
    if constexpr (NF == 0)  // no medium
        return args.med.spot ? launch_mixed_nf<NF, true, 3>(args, L, grid, st)
                             : launch_mixed_nf<NF, true, 1>(args, L, grid, st);
    else if (!args.single_medium)
        return launch_mixed_nf<NF, false, 0>(args, L, grid, st);
    else
        return args.med.synch ? launch_mixed_nf<NF, true, 2>(args, L, grid, st)
                              : launch_mixed_nf<NF, true, 1>(args, L, grid, st);
}

// The tracing kernel for NF transfer slots, instantiated in trace_mixed_nf<NF>.cu.
extern template cudaError_t launch_mixed_nf<0>(const TraceArgs &, const odx_launch &, dim3, cudaStream_t);
extern template cudaError_t launch_mixed_nf<3>(const TraceArgs &, const odx_launch &, dim3, cudaStream_t);
extern template cudaError_t launch_mixed_nf<4>(const TraceArgs &, const odx_launch &, dim3, cudaStream_t);
extern template cudaError_t launch_mixed_nf<8>(const TraceArgs &, const odx_launch &, dim3, cudaStream_t);

}  // namespace odx
