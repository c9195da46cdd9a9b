// Kernels of the GB300 lattice Boltzmann step (templates; instantiated per
// storage format in lbm_kernels_<format>.cu).
//
//  step_kernel      fused stream + collide for one A-A half of the pattern:
//                   one read and one write per population, boundary rules
//                   and the moving lid folded into the addressing; LBGK,
//                   ELBM, positivity and MRT are complete here, the Ehrenfest
//                   and median limiters additionally append their candidate
//                   sites (Delta S > delta) to a compact list.
//  ehrenfest_eval_select  the side of delta of each screened site, settled
//                   in FP32 where the error bound allows, else by its FP64
//                   Delta S; then the k-largest selection (ranks, or an MSB
//                   radix select on the FP64 Delta S bits in the last CTA),
//                   ties by site index; selected sites are rewritten with f*.
//  median_fixup     grid-stride over candidates: median of the Delta S window
//                   (a field the step wrote), homothety of Eq. (entrHom)
//                   where it lowers Delta S.
//  median_recon_fixup  the same without a field: the window's Delta S from
//                   the pre-collision state recovered from the LBGK
//                   post-collision one (FP32 / FP64 storage).
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int kBlockX = 128;
constexpr int kBlockY = 2;

// Programmatic dependent launch: a step kernel may be launched while the
// previous kernel of the stream finishes its last wave.  Every kernel so
// launched waits, before its first global memory access, until the previous
// grid has completed and its writes are visible; each CTA then allows the
// next kernel to launch (it starts once every CTA of this grid has started).
// Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ int lane_id() {
    return (threadIdx.y * blockDim.x + threadIdx.x) & 31;
}

// Appends a screened site (Delta S possibly above delta) to the compact list:
// its pre-collision populations and site index.  Such sites are rare, so one
// atomic each; a full list sets the overflow flag.  The FP64 Delta S is
// evaluated afterwards by eval_kernel / median_fixup, off the streaming path.
template <int Q, class T>
struct Pops {
    T v[Q];
};

// The side of delta a screened site's Delta S is on, where FP32 arithmetic
// settles it: the site's FP32 Delta S (delta_s_and_q, the median screen's
// evaluation) lies within 1e-3 relative plus 1e-6 sqrt(q rho) of the exact
// value (the bound the screens use), so 1 = certainly above delta, 0 =
// certainly not, 2 = too close (or non-finite): the FP64 value decides.
// Used by the selection kernel on the recorded populations.
template <int Q>
__device__ __forceinline__ int certify_side(const Params& p, const float* f, float& ds) {
    float rho, ux, uy, feq[Q], q;
    moments<Q, float>(f, rho, ux, uy);
    equilibrium<Q, float>(p.eq, rho, ux, uy, feq);
    ds = delta_s_and_q<Q, float>(f, feq, q);
    if (!(ds < INFINITY)) return 2;
    const float s = 1e-6f * sqrtf(fabsf(q * rho));
    if ((double)(0.999f * ds - s) > p.delta) return 1;
    if ((double)(1.001f * ds + s) <= p.delta) return 0;
    return 2;
}

// Out of line: the call is rare, and its address arithmetic and stores stay
// out of the streaming path's register allocation.
template <int Q, class T>
__device__ __noinline__ void record_candidate_cold(const Params& p, int site, Pops<Q, T> f) {
    const unsigned pos = atomicAdd(&p.counters[p.cslot], 1u);
    if (pos < (unsigned)p.cand_cap) {
        T* cf = (T*)p.cand_f;
#pragma unroll
        for (int i = 0; i < Q; ++i) cf[(int64_t)i * p.cand_cap + pos] = f.v[i];
        p.cand_site[pos] = site;
    } else {
        atomicExch(&p.counters[CNT_OVERFLOW], 1u);
    }
}

template <int Q, class T>
__device__ __forceinline__ void record_candidate(const Params& p, int x, int y, const T* f) {
    Pops<Q, T> v;
#pragma unroll
    for (int i = 0; i < Q; ++i) v.v[i] = f[i];
    record_candidate_cold<Q, T>(p, y * p.nx + x, v);
}

// Limiter screen of the pre-collision state: the sites that may exceed
// delta (FP32 screens of Eq. DelS) are appended to the candidate list; their
// FP64 value decides later.  The median filter with a Delta S field also
// writes every site's Delta S there (in the arithmetic type; FP64 in FP64
// mode); without the field the median step screens like the Ehrenfest one.
template <int Q, class T, int COLL>
__device__ __forceinline__ void limiter_screen(const Params& p, int x, int y, const T* f,
                                               const T* feq, T rho) {
    bool maybe;
    if (COLL == LBM_MEDIAN) {
        T q;
        const T ds = delta_s_and_q<Q, T>(f, feq, q);
        ((T*)p.ds_field)[(int64_t)y * p.nx + x] = ds;
        maybe = median_maybe_above((float)ds, (float)q, (float)rho, p.delta_f);
    } else {
        float ff[Q], fq[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            ff[i] = (float)f[i];
            fq[i] = (float)feq[i];
        }
        maybe = maybe_above_loose<Q>(ff, fq, (float)rho, p.delta_f);
    }
    if (maybe) record_candidate<Q, T>(p, x, y, f);
}

// Collision of one site, pre-collision f to post-collision F: moments,
// divergence check, equilibrium, limiter screen, collision, exact mass.
template <int Q, class ST, int COLL>
__device__ __forceinline__ void collide_site(const Params& p, int x, int y, const typename ST::T* f,
                                             typename ST::T* F, int& e_code, int& e_iters,
                                             typename ST::T& acc) {
    using T = typename ST::T;
    T rho, ux, uy;
    moments<Q, T>(f, rho, ux, uy);
    // once set the flag is only read: a diverged lattice would otherwise
    // send every site's atomic to one address
    if (!(rho > T(0)) || !(fabs(ux) < T(1e30)) || !(fabs(uy) < T(1e30)))
        if (*(volatile unsigned*)&p.counters[CNT_DIVERGED] == 0u) atomicExch(&p.counters[CNT_DIVERGED], 1u);
    if (COLL == LBM_ELBM) {
        double fd[Q], fe[Q], Dd[Q], r, a, b;
#pragma unroll
        for (int i = 0; i < Q; ++i) fd[i] = (double)f[i];
        moments<Q, double>(fd, r, a, b);
        equilibrium<Q, double>(LBM_EQ_ENTROPIC, r, a, b, fe);
#pragma unroll
        for (int i = 0; i < Q; ++i) Dd[i] = fe[i] - fd[i];
        ElbmOut out = elbm_alpha<Q>(fd, fe, Dd, r, p);
        e_code = out.code;
        e_iters = out.iters;
        const double ab = out.alpha * p.beta;
        if constexpr (sizeof(T) == 8) {
#pragma unroll
            for (int i = 0; i < Q; ++i) F[i] = fd[i] + ab * Dd[i];
        } else {
            // F = f + alpha beta (f* - f) rounds to FP32 (or 16 bits) anyway:
            // the product in FP32 on the FP64 difference, no FP64 update
            const float abf = (float)ab;
#pragma unroll
            for (int i = 0; i < Q; ++i) F[i] = fmaf(abf, (float)Dd[i], f[i]);
        }
    } else if ((COLL >= LBM_SMOOTH && COLL <= LBM_THRESHOLD) || COLL == LBM_ENSEMBLE_LAGGED) {
        // Sections 4.2-4.4: f -> f* + phi(Delta S) (f - f*), then LBGK, i.e.
        // F = f* + (1 - 2 beta) phi (f - f*); the threshold limiter's phi is
        // decided after the step (the sites above Delta S_t are rewritten)
        T feq[Q], q;
        equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
        const T ds = delta_s_and_q<Q, T>(f, feq, q);
        T phi = T(1);
        if (COLL == LBM_ENSEMBLE_LAGGED && isfinite(ds)) {
            acc += ds;  // the next step's E: this step's sum and count
            e_code = 1;
        }
        if (COLL == LBM_THRESHOLD) {
            if (isfinite(ds)) acc += ds;  // the step's sum of Delta S
            if (median_maybe_above((float)ds, (float)q, (float)rho, p.delta_f)) record_candidate<Q, T>(p, x, y, f);
        } else if (!(ds < T(INFINITY))) {
            phi = T(0);  // a negative population: the state goes to f*
        } else {
            constexpr bool d = sizeof(T) == 8;  // FP64 parameters, else their FP32 copies
            const T alpha = d ? T(p.lim_alpha) : T(p.lim_f[0]), k = d ? T(p.lim_k) : T(p.lim_f[1]);
            if (COLL == LBM_SMOOTH) {
                phi = T(1) / (T(1) + alpha * pow_lim(ds, k));
            } else if (COLL == LBM_DOUBLE_MONOTONIC) {
                const T z = d ? ds / T(p.lim_dst) : ds * T(p.lim_f[2]);
                phi = pow_lim(T(1) + pow_lim(z, k), d ? T(-0.5) / k : T(p.lim_f[3]));
            } else {  // LBM_ENSEMBLE (E from this step's pre-pass), LBM_ENSEMBLE_LAGGED (the previous step's)
                const T E = d ? T(*p.lim_E) : T(*p.lim_E_f);
                if (E > T(0)) {
                    const T yv = ds / (alpha * E);
                    phi = (T(1) + pow_lim(yv, k - T(0.5))) / (T(1) + pow_lim(yv, k));
                }
            }
        }
        const T c = (T(1) - (sizeof(T) == 8 ? T(2.0 * p.beta) : T(2) * T(p.beta_f))) * phi;
#pragma unroll
        for (int i = 0; i < Q; ++i) F[i] = feq[i] + c * (f[i] - feq[i]);
    } else {
        T feq[Q];
        equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
        if (COLL == LBM_EHRENFEST || COLL == LBM_MEDIAN || COLL == LBM_MRT_LIMITER)
            limiter_screen<Q, T, COLL == LBM_MRT_LIMITER ? LBM_EHRENFEST : COLL>(p, x, y, f, feq, rho);
        if (COLL == LBM_MRT && Q == 9) {
            mrt_d2q9<T>(f, feq, p.mrt, p.mrt_f, F);
        } else if (COLL == LBM_MRT2 && Q == 9) {
            mrt2_d2q9<T>(f, feq, sizeof(T) == 8 ? T(2.0 * p.beta) : T(2) * T(p.beta_f), F);
        } else {
            lbgk<Q, T>(f, feq, sizeof(T) == 8 ? T(p.beta) : T(p.beta_f), F);
        }
        if (COLL == LBM_POSITIVITY) {
            if (positivity<Q, T>(feq, F)) atomicAdd(&p.stats[ST_LIMITED], 1ull);
        }
    }
    conserve_mass<Q, T>(rho, F);
}

// The same collision in deviation form for the 16-bit formats, whose stored
// value is the deviation d_i = f_i - W_i: with sum_i W_i = 1 and
// sum_i W_i v_i = 0, rho = 1 + sum_i d_i and rho u = sum_i v_i d_i; the
// equilibrium enters as d*_i = f*_i - W_i, and LBGK, MRT and A_2 only use
// differences f - f* = d - d*, so the post-collision deviation
// D_i = F_i - W_i comes out directly (no W_i added on load or subtracted on
// store).  The Ehrenfest screen and the positivity rule form absolute values
// where they need them.  D2Q9, the collisions of the paired kernel, for one
// site (V = float) or two adjacent sites at once (V = F2, the pair kernel):
// the same operations in the same order, so either form gives the same bits.
// The per-lane parts (the division by rho, the tests, the rare candidate
// record and positivity fix-up) run on each lane's value.
//
// Equilibrium d*_i; with MIN also a lower bound of min_i f*_i per lane for
// the limiter screen: for the product equilibria the product of the 1D
// minima when every factor is positive (else 0, which passes every site to
// the exact test).
template <class V, bool MIN>
__device__ __forceinline__ void equilibrium_dev9(int kind, V drho, V rho, V ux, V uy, V* ds, float* m) {
    using L = Lat<9>;
    constexpr int NL = VLanes<V>::n;
    const V one = vsplat(1.f, rho);
    if (kind == LBM_EQ_POLY_STD) {
        // textbook form: d*_i = W_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 u^2))
        const V nuu = vmul(vsplat(-1.5f, rho), vfma(ux, ux, vmul(uy, uy)));
        V rest = drho;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const V cu = vfma(vsplat(float(L::cx(i)), rho), ux, vmul(vsplat(float(L::cy(i)), rho), uy));
            const V a = vfma(vmul(vsplat(4.5f, rho), cu), cu, vfma(vsplat(3.f, rho), cu, nuu));
            ds[i] = vmul(vsplat(float(L::w(i)), rho), vfma(rho, a, drho));
            rest = vsub(rest, ds[i]);
        }
        ds[0] = rest;
        if (MIN) {
            // min f*, 0 when not positive
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                float mk = float(L::w(0)) + vlane(rest, k);
#pragma unroll
                for (int i = 1; i < 9; ++i) mk = fminf(mk, float(L::w(i)) + vlane(ds[i], k));
                m[k] = fmaxf(mk, 0.f);
            }
        }
        return;
    }
    // product of the 1D factors a_-, a_0, a_+ = a - u/2, 1 - 2a, a + u/2
    V ax[3], ay[3];
    const V uv[2] = {ux, uy};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const V u = uv[c];
        const V t = vfma(vmul(vsplat(3.f, rho), u), u, one);  // 1 + 3 u^2
        V a;
        if (kind == LBM_EQ_ENTROPIC) {
            float sq[NL];
#pragma unroll
            for (int k = 0; k < NL; ++k) sq[k] = __fsqrt_rn(vlane(t, k));
            a = vmul(vfma(vsplat(2.f, rho), vmake<V>(sq[0], sq[NL - 1]), vsplat(-1.f, rho)), vsplat(1.f / 6.f, rho));
        } else {
            a = vmul(t, vsplat(1.f / 6.f, rho));
        }
        const V h = vmul(vsplat(0.5f, rho), u);
        V* f1 = c == 0 ? ax : ay;
        f1[0] = vsub(a, h);
        f1[1] = vfma(vsplat(-2.f, rho), a, one);
        f1[2] = vadd(a, h);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) ax[k] = vmul(ax[k], rho);
    if (MIN) {
        // min f* = (min of the rho-scaled x factors) (min of the y factors),
        // 0 when either is not positive
        float mx[NL], my[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            mx[k] = fmaxf(fminf(fminf(vlane(ax[0], k), vlane(ax[1], k)), vlane(ax[2], k)), 0.f);
            my[k] = fmaxf(fminf(fminf(vlane(ay[0], k), vlane(ay[1], k)), vlane(ay[2], k)), 0.f);
        }
        const V mv = vmul(vmake<V>(mx[0], mx[NL - 1]), vmake<V>(my[0], my[NL - 1]));
#pragma unroll
        for (int k = 0; k < NL; ++k) m[k] = vlane(mv, k);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) ds[i] = vfma(ax[L::cx(i) + 1], ay[L::cy(i) + 1], vsplat(-float(L::w(i)), rho));
}

// MRT of Section 5 (mrt_d2q9: M1's orthogonal rows, rest, E, SE, S, SW, W,
// NW, N, NE numbering) in deviation form on e = f - f*: the non-conserved
// moments of e scaled by C1 N^-1 (rates), then D = d - M1^T m.  Explicit
// operations for one site or a pair (the same bits either way).
template <class V>
__device__ __forceinline__ void mrt_dev(const V* d, const V* e, const MrtRatesF& r, V* D) {
    const V se = vadd(vadd(e[2], e[4]), vadd(e[6], e[8]));  // diagonals
    const V ax = vadd(vadd(e[1], e[3]), vadd(e[5], e[7]));  // axis
    const V two = vsplat(2.f, se), four = vsplat(4.f, se), mtwo = vsplat(-2.f, se);
    // e_m = -4 e0 - ax + 2 se, eps_m = 4 e0 - 2 ax + se
    const V em = vmul(vsub(vfma(two, se, vmul(vsplat(-4.f, se), e[0])), ax), vsplat(r.e, se));
    const V ep = vmul(vadd(vfma(mtwo, ax, vmul(four, e[0])), se), vsplat(r.eps, se));
    // q_x = -2 e1 + e2 - e4 + 2 e5 - e6 + e8, q_y = -e2 + 2 e3 - e4 + e6 - 2 e7 + e8
    const V qx = vmul(vfma(two, vsub(e[5], e[1]), vadd(vsub(e[2], e[4]), vsub(e[8], e[6]))), vsplat(r.q, se));
    const V qy = vmul(vfma(two, vsub(e[3], e[7]), vadd(vsub(e[6], e[2]), vsub(e[8], e[4]))), vsplat(r.q, se));
    // p_xx = e1 - e3 + e5 - e7, p_xy = -e2 + e4 - e6 + e8
    const V pxx = vmul(vsub(vadd(e[1], e[5]), vadd(e[3], e[7])), vsplat(r.nu, se));
    const V pxy = vmul(vsub(vadd(e[4], e[8]), vadd(e[2], e[6])), vsplat(r.nu, se));
    const V a = vfma(mtwo, ep, vsub(vsplat(0.f, se), em));  // -e - 2 eps (axis rows)
    const V b = vfma(two, em, ep);                           // 2 e + eps (diagonal rows)
    D[0] = vsub(d[0], vmul(four, vsub(ep, em)));
    D[1] = vsub(d[1], vadd(vfma(mtwo, qx, a), pxx));
    D[2] = vsub(d[2], vsub(vadd(b, vsub(qx, qy)), pxy));
    D[3] = vsub(d[3], vsub(vfma(two, qy, a), pxx));
    D[4] = vsub(d[4], vadd(vsub(b, vadd(qx, qy)), pxy));
    D[5] = vsub(d[5], vadd(vfma(two, qx, a), pxx));
    D[6] = vsub(d[6], vsub(vadd(b, vsub(qy, qx)), pxy));
    D[7] = vsub(d[7], vsub(vfma(mtwo, qy, a), pxx));
    D[8] = vsub(d[8], vadd(vadd(b, vadd(qx, qy)), pxy));
}

// One site (V = float): a screened site is recorded as a candidate.  Two
// sites (V = F2): nothing is recorded; bit k of *scr is set when site k
// needs the record, and the caller runs both sites again through the
// one-site form (the same operations, so the same result), which records.
// (Keeping the pre-collision state live for the rare record would hold 18
// more registers through the collision.)
template <class V, class ST, int COLL>
__device__ __forceinline__ void collide_dev(const Params& p, int x, int y, const V* d, V* D,
                                            unsigned* scr = nullptr) {
    using L = Lat<9>;
    constexpr int NL = VLanes<V>::n;
    constexpr bool kScreen = COLL == LBM_EHRENFEST || COLL == LBM_MRT_LIMITER;
    static_assert(L::cx(1) == 1 && L::cx(2) == 1 && L::cx(8) == 1 && L::cx(4) == -1 && L::cx(5) == -1 &&
                      L::cx(6) == -1 && L::cy(6) == 1 && L::cy(7) == 1 && L::cy(8) == 1 && L::cy(2) == -1 &&
                      L::cy(3) == -1 && L::cy(4) == -1,
                  "D2Q9 numbering of Lat<9>");
    V drho = d[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) drho = vadd(drho, d[i]);
    const V jx = vsub(vadd(vadd(d[1], d[2]), d[8]), vadd(vadd(d[4], d[5]), d[6]));
    const V jy = vsub(vadd(vadd(d[6], d[7]), d[8]), vadd(vadd(d[2], d[3]), d[4]));
    const V rho = vadd(vsplat(1.f, drho), drho);
    float inv[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) inv[k] = __fdiv_rn(1.f, vlane(rho, k));
    const V vinv = vmake<V>(inv[0], inv[NL - 1]);
    const V ux = vmul(jx, vinv), uy = vmul(jy, vinv);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NL; ++k)
        bad |= !(vlane(rho, k) > 0.f) || !(fabsf(vlane(ux, k)) < 1e30f) || !(fabsf(vlane(uy, k)) < 1e30f);
    if (bad)
        if (*(volatile unsigned*)&p.counters[CNT_DIVERGED] == 0u) atomicExch(&p.counters[CNT_DIVERGED], 1u);
    V ds[9], e[9];
    float m[NL];
    equilibrium_dev9<V, kScreen>(p.eq, drho, rho, ux, uy, ds, m);
    V s2;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        e[i] = vsub(d[i], ds[i]);  // f - f*
        if (kScreen) s2 = i == 0 ? vmul(e[0], e[0]) : vfma(e[i], e[i], s2);
        if (COLL == LBM_EHRENFEST || COLL == LBM_MRT_LIMITER) D[i] = vfma(vsplat(-2.f * p.beta_f, rho), e[i], d[i]);
    }
    if (kScreen) {
        // The screen of maybe_above_loose on f - f* with m a lower bound of
        // min f* (the bound's argument holds for any positive one), first as
        // one product test without the division: a site is quiet when
        // s2 < m min(m / 4, 0.998 delta) and rho < 1e6 delta.  Then
        // Delta S <= s2 / m < 0.998 delta, and the FP32 rounding of f* and
        // d (at most 2e-6 q + 3e-7 sqrt(q rho)) stays inside the 0.2% margin
        // for rho < 4e7 delta.
        const float dq = 0.998f * p.delta_f, rq = 1e6f * p.delta_f;
        // (m = 0 when f* has a non-positive population: bound 0, never quiet)
        const V mv = vmake<V>(m[0], m[NL - 1]);
        const V m4 = vmul(mv, vsplat(0.25f, mv));
        float lim[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) lim[k] = fminf(vlane(m4, k), dq);
        const V bound = vmul(mv, vmake<V>(lim[0], lim[NL - 1]));
        unsigned mask = 0u;
#pragma unroll
        for (int k = 0; k < NL; ++k)
            if (!(vlane(s2, k) < vlane(bound, k) && vlane(rho, k) < rq)) mask |= 1u << k;
        if (mask) {
            // not certified quiet (near delta, a tiny delta, or not finite):
            // the division form of the same screen decides
#pragma unroll
            for (int k = 0; k < NL; ++k) {
                const float s2k = vlane(s2, k), mk = m[k];
                if ((mask >> k & 1u) && mk > 0.f && s2k < 0.25f * mk * mk &&
                    !slack_reaches(__fdividef(s2k, mk), __fdividef(s2k, mk), vlane(rho, k), p.delta_f))
                    mask &= ~(1u << k);
            }
        }
        if constexpr (NL == 1) {
            if (mask) {
                const unsigned pos = atomicAdd(&p.counters[p.cslot], 1u);
                if (pos < (unsigned)p.cand_cap) {
                    float* cf = (float*)p.cand_f + pos;
#pragma unroll
                    for (int i = 0; i < 9; ++i) cf[(int64_t)i * p.cand_cap] = float(L::w(i)) + vlane(d[i], 0);
                    p.cand_site[pos] = y * p.nx + x;
                } else {
                    atomicExch(&p.counters[CNT_OVERFLOW], 1u);
                }
            }
        } else {
            *scr = mask;
        }
    }
    const float om = 2.f * p.beta_f;
    if (COLL == LBM_MRT) {
        mrt_dev<V>(d, e, p.mrt_f, D);
    } else if (COLL == LBM_MRT2) {
        // A_2: D = d* + (1 - s_nu)/4 (m4 r4 + m5 r5), m = r . (f - f*)
        const V c = vsplat((1.f - om) * 0.25f, rho);
        const V m4 = vmul(vsub(vadd(e[1], e[5]), vadd(e[3], e[7])), c);
        const V m5 = vmul(vsub(vadd(e[4], e[8]), vadd(e[2], e[6])), c);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int r4 = L::cx(i) * L::cx(i) - L::cy(i) * L::cy(i), r5 = L::cx(i) * L::cy(i);
            D[i] = r4 > 0 ? vadd(ds[i], m4) : r4 < 0 ? vsub(ds[i], m4) : r5 > 0 ? vadd(ds[i], m5)
                                                     : r5 < 0 ? vsub(ds[i], m5) : ds[i];
        }
    } else if (COLL != LBM_EHRENFEST && COLL != LBM_MRT_LIMITER) {
        // LBGK: F = f - 2 beta (f - f*)
        const V nom = vsplat(-om, rho);
#pragma unroll
        for (int i = 0; i < 9; ++i) D[i] = vfma(nom, e[i], d[i]);
    }
    if (COLL == LBM_POSITIVITY && NL > 1) {
        // a negative population (rare): the caller runs both sites again
        // through the one-site form, which applies the rule
        unsigned mask = 0u;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            bool neg = false;
#pragma unroll
            for (int i = 0; i < 9; ++i) neg |= vlane(D[i], k) < -float(L::w(i));
            if (neg) mask |= 1u << k;
        }
        *scr = mask;
    } else if (COLL == LBM_POSITIVITY) {
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            bool neg = false;
#pragma unroll
            for (int i = 0; i < 9; ++i) neg |= vlane(D[i], k) < -float(L::w(i));
            if (neg) {
                float fe[9], F[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    fe[i] = float(L::w(i)) + vlane(ds[i], k);
                    F[i] = float(L::w(i)) + vlane(D[i], k);
                }
                if (positivity<9, float>(fe, F)) atomicAdd(&p.stats[ST_LIMITED], 1ull);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const float v = F[i] - float(L::w(i));
                    D[i] = vmake<V>(k == 0 ? v : vlane(D[i], 0), k == 0 ? vlane(D[i], NL - 1) : v);
                }
            }
        }
    }
    // every collision conserves mass: the rest population as rho minus the others
    V sD = D[1];
#pragma unroll
    for (int i = 2; i < 9; ++i) sD = vadd(sD, D[i]);
    D[0] = vsub(drho, sD);
}

// ---------------------------------------------------------------------------
// The Section 4.2-4.4 limiters on D2Q9 in FP32 arithmetic (FP32 and 16-bit
// storage), one site per thread: moments, the equilibrium and Delta S as
// explicit correctly rounded operations (nothing left to contraction) with
// one approximate reciprocal per population, then phi per site.  (On packed
// pairs, two sites per thread, the step needs ~116 registers, two CTAs per
// SM, and measured slower.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// rho, u and f* (absolute) of D2Q9 populations f
__device__ __forceinline__ void lim_state(int kind, const float* f, float& rho, float& ux, float& uy,
                                          float* feq) {
    using L = Lat<9>;
    static_assert(L::cx(1) == 1 && L::cx(2) == 1 && L::cx(8) == 1 && L::cx(4) == -1 && L::cx(5) == -1 &&
                      L::cx(6) == -1 && L::cy(6) == 1 && L::cy(7) == 1 && L::cy(8) == 1 && L::cy(2) == -1 &&
                      L::cy(3) == -1 && L::cy(4) == -1,
                  "D2Q9 numbering of Lat<9>");
    rho = f[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) rho = __fadd_rn(rho, f[i]);
    const float jx = __fsub_rn(__fadd_rn(__fadd_rn(f[1], f[2]), f[8]), __fadd_rn(__fadd_rn(f[4], f[5]), f[6]));
    const float jy = __fsub_rn(__fadd_rn(__fadd_rn(f[6], f[7]), f[8]), __fadd_rn(__fadd_rn(f[2], f[3]), f[4]));
    const float inv = __fdiv_rn(1.f, rho);
    ux = __fmul_rn(jx, inv);
    uy = __fmul_rn(jy, inv);
    if (kind == LBM_EQ_POLY_STD) {
        const float nuu = __fmul_rn(-1.5f, __fmaf_rn(ux, ux, __fmul_rn(uy, uy)));
        float rest = rho;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float cu = __fmaf_rn(float(L::cx(i)), ux, __fmul_rn(float(L::cy(i)), uy));
            const float a = __fmaf_rn(__fmul_rn(4.5f, cu), cu, __fmaf_rn(3.f, cu, nuu));
            feq[i] = __fmul_rn(float(L::w(i)), __fmaf_rn(rho, a, rho));
            rest = __fsub_rn(rest, feq[i]);
        }
        feq[0] = rest;
        return;
    }
    // product of the 1D factors a_-, a_0, a_+ = a - u/2, 1 - 2a, a + u/2
    float ax[3], ay[3];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float u = c == 0 ? ux : uy;
        const float t = __fmaf_rn(__fmul_rn(3.f, u), u, 1.f);  // 1 + 3 u^2
        const float a = kind == LBM_EQ_ENTROPIC ? __fmul_rn(__fmaf_rn(2.f, __fsqrt_rn(t), -1.f), 1.f / 6.f)
                                                : __fmul_rn(t, 1.f / 6.f);
        const float h = __fmul_rn(0.5f, u);
        float* f1 = c == 0 ? ax : ay;
        f1[0] = __fsub_rn(a, h);
        f1[1] = __fmaf_rn(-2.f, a, 1.f);
        f1[2] = __fadd_rn(a, h);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) ax[k] = __fmul_rn(ax[k], rho);
#pragma unroll
    for (int i = 0; i < 9; ++i) feq[i] = __fmul_rn(ax[L::cx(i) + 1], ay[L::cy(i) + 1]);
}

// sum_i dx_i P_K(x_i), P_K the series of g(x) / x^2 (gpoly_f's coefficients)
template <int K>
__device__ __forceinline__ float lim_series(const float* dx, const float* x) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        float pk = ((K & 1) ? -1.0f : 1.0f) / (float)((K + 1) * (K + 2));
#pragma unroll
        for (int k = K - 1; k >= 0; --k) pk = __fmaf_rn(pk, x[i], ((k & 1) ? -1.0f : 1.0f) / (float)((k + 1) * (k + 2)));
        s = i == 0 ? __fmul_rn(dx[0], pk) : __fmaf_rn(dx[i], pk, s);
    }
    return s;
}

// Delta S (Eq. DelS, the FP32 screen evaluation) and q = sum (f - f*)^2 / f*:
// one series length per site, chosen by max |x| (the tiers of
// delta_s_and_q<9, float>), the closed form g(x) = (1 + x) ln(1 + x) - x
// beyond 1/4; +inf with a non-positive f* or population.
__device__ __forceinline__ float delta_s_lim(const float* f, const float* feq, float& q) {
    float x[9], dx[9], amax = 0.f, emin = feq[0];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float d = __fsub_rn(f[i], feq[i]);
        x[i] = __fmul_rn(d, rcp_approx(feq[i]));
        dx[i] = __fmul_rn(d, x[i]);
        amax = fmaxf(amax, fabsf(x[i]));
        emin = fminf(emin, feq[i]);
    }
    q = dx[0];
#pragma unroll
    for (int i = 1; i < 9; ++i) q = __fadd_rn(q, dx[i]);
    if (!(emin > 0.f)) return INFINITY;
    if (amax < 0x1p-12f) return lim_series<1>(dx, x);
    if (amax < 0.03125f) return lim_series<4>(dx, x);
    if (amax < 0.25f) return lim_series<11>(dx, x);
    float s = 0.f;
    bool neg = false;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        neg |= f[i] < 0.f;
        s = fmaf(feq[i], gfun_f(x[i]), s);
    }
    return neg ? INFINITY : s;
}

// The collision: F = f* + (1 - 2 beta) phi (f - f*) (c27), phi from the
// site's Delta S; the threshold limiter keeps phi = 1 here and screens
// candidates, its rewrite follows the step; the threshold and lagged-ensemble
// limiters add a finite Delta S to acc (cnt counts it).
template <int COLL>
__device__ __forceinline__ void collide_lim(const Params& p, int x, int y, const float* f, float* F, float& acc,
                                            int& cnt) {
    float rho, ux, uy, feq[9], q;
    lim_state(p.eq, f, rho, ux, uy, feq);
    if (!(rho > 0.f) || !(fabsf(ux) < 1e30f) || !(fabsf(uy) < 1e30f))
        if (*(volatile unsigned*)&p.counters[CNT_DIVERGED] == 0u) atomicExch(&p.counters[CNT_DIVERGED], 1u);
    const float ds = delta_s_lim(f, feq, q);
    float phi = 1.f;
    if ((COLL == LBM_ENSEMBLE_LAGGED || COLL == LBM_THRESHOLD) && isfinite(ds)) {
        acc += ds;
        ++cnt;
    }
    if (COLL == LBM_THRESHOLD) {
        if (median_maybe_above(ds, q, rho, p.delta_f)) record_candidate<9, float>(p, x, y, f);
    } else if (!(ds < INFINITY)) {
        phi = 0.f;  // a negative population: the state goes to f*
    } else {
        // approximate divisions (2 ulp): phi only scales the non-equilibrium part
        const float alpha = p.lim_f[0], k = p.lim_f[1];
        if (COLL == LBM_SMOOTH) {
            phi = __fdividef(1.f, 1.f + alpha * pow_lim(ds, k));
        } else if (COLL == LBM_DOUBLE_MONOTONIC) {
            phi = pow_lim(1.f + pow_lim(ds * p.lim_f[2], k), p.lim_f[3]);
        } else {  // LBM_ENSEMBLE, LBM_ENSEMBLE_LAGGED
            const float E = *p.lim_E_f;
            if (E > 0.f) {
                const float yv = __fdividef(ds, alpha * E);
                phi = __fdividef(1.f + pow_lim(yv, k - 0.5f), 1.f + pow_lim(yv, k));
            }
        }
    }
    const float c = (1.f - 2.f * p.beta_f) * phi;
#pragma unroll
    for (int i = 0; i < 9; ++i) F[i] = __fmaf_rn(c, __fsub_rn(f[i], feq[i]), feq[i]);
    // every collision conserves mass: the rest population as rho minus the others
    float sF = F[1];
#pragma unroll
    for (int i = 2; i < 9; ++i) sF = __fadd_rn(sF, F[i]);
    F[0] = __fsub_rn(rho, sF);
}

// Section 8's diffusive Maxwell rule at wall site (x, y) (bc DIFFUSIVE), on
// its pre-collision populations: at a site of one wall (outward normal n)
// the populations with v . n < 0 become gamma f*_i(u_wall), f* at unit
// density, gamma = sum_{v.n > 0} f_j / sum_{v.n < 0} f*_i; at a corner each
// population from outside the box takes its opposite's value when that
// one came from inside (the rule with a single population: bounce-back).
template <class T>
__device__ __forceinline__ void diffusive_rule(const Params& p, int x, int y, T* f) {
    using L = Lat<9>;
    const int nxw = (x == 0 ? -1 : 0) + (x == p.nx - 1 ? 1 : 0);
    const int nyw = (y == 0 ? -1 : 0) + (y == p.ny - 1 ? 1 : 0);
    if (nxw != 0 && nyw != 0) {
        T g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = f[i];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = x - L::cx(i), sy = y - L::cy(i);
            const int o = L::opp(i), ox = x - L::cx(o), oy = y - L::cy(o);
            const bool out_i = sx < 0 || sx >= p.nx || sy < 0 || sy >= p.ny;
            const bool in_o = ox >= 0 && ox < p.nx && oy >= 0 && oy < p.ny;
            if (out_i && in_o) f[i] = g[o];
        }
        return;
    }
    T feq[9];
    const T uw = nyw == 1 ? T(p.wall_u) : T(0);
    equilibrium<9, T>(p.eq, T(1), uw, T(0), feq);
    T out = T(0), in = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int vn = L::cx(i) * nxw + L::cy(i) * nyw;
        if (vn > 0) out += f[i];
        if (vn < 0) in += feq[i];
    }
    const T gamma = out / in;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (L::cx(i) * nxw + L::cy(i) * nyw < 0) f[i] = gamma * feq[i];
}

// The whole step for the site (x, y): load (streaming in odd steps),
// collision, store.
// The 16-bit D2Q9 collisions that run in deviation form (collide_dev),
// at every site so that every kernel computes a site alike.
template <int Q, class ST, int COLL>
constexpr bool kDeviationForm = Q == 9 && sizeof(typename ST::S) == 2 &&
                                (COLL == LBM_LBGK || COLL == LBM_EHRENFEST || COLL == LBM_POSITIVITY ||
                                 COLL == LBM_MRT || COLL == LBM_MRT2 || COLL == LBM_MRT_LIMITER);

// The D2Q9 Section 4.2-4.4 limiters in FP32 arithmetic (FP32 and 16-bit
// storage) that run collide_lim, at every site so that every kernel computes
// a site alike.
template <int Q, class ST, int COLL>
constexpr bool kLimForm = Q == 9 && sizeof(typename ST::T) == 4 &&
                          (COLL == LBM_SMOOTH || COLL == LBM_DOUBLE_MONOTONIC || COLL == LBM_ENSEMBLE ||
                           COLL == LBM_THRESHOLD || COLL == LBM_ENSEMBLE_LAGGED);

template <int Q, class ST, int COLL, bool ODD>
__device__ __forceinline__ void site_update(const Params& p, int x, int y, int& e_code,
                                            int& e_iters, typename ST::T& acc) {
    using T = typename ST::T;
    constexpr bool DEV = kDeviationForm<Q, ST, COLL>;
    T f[Q], F[Q];
    const bool interior = x > 0 && x < p.nx - 1 && (Q == 3 || (y > 0 && y < p.ny - 1));
    const int o = y * p.pitch + x;
    if (interior) {
        load_interior<Q, ST, ODD, DEV>(p, o, f);
    } else {
        // diffusive walls: wall sites are updated by diffusive_wall_kernel
        // (each site owns its addresses, so the two kernels of a step commute)
        if (Q == 9 && p.diffusive) return;
        load_general<Q, ST, ODD, DEV>(p, x, y, f);
    }
    if constexpr (DEV) {
        collide_dev<float, ST, COLL>(p, x, y, f, F);
    } else if constexpr (kLimForm<Q, ST, COLL>) {
        float a = 0.f;
        int cnt = 0;
        collide_lim<COLL>(p, x, y, f, F, a, cnt);
        acc += a;
        if (cnt) e_code = 1;
    } else {
        collide_site<Q, ST, COLL>(p, x, y, f, F, e_code, e_iters, acc);
    }
    if (interior)
        store_interior<Q, ST, ODD, DEV>(p, o, F);
    else
        store_general<Q, ST, ODD, DEV>(p, x, y, F);
}

// Warp-aggregated ELBM counters (all 32 lanes of the warp call this).
__device__ __forceinline__ void elbm_stats(const Params& p, int e_code, int e_iters) {
    unsigned solved = __reduce_add_sync(0xffffffffu, e_code == 0 ? 1u : 0u);
    unsigned skipped = __reduce_add_sync(0xffffffffu, e_code == 1 ? 1u : 0u);
    unsigned fallback = __reduce_add_sync(0xffffffffu, e_code == 2 ? 1u : 0u);
    unsigned iters = __reduce_add_sync(0xffffffffu, (unsigned)e_iters);
    unsigned itmax = __reduce_max_sync(0xffffffffu, (unsigned)e_iters);
    if (lane_id() == 0) {
        if (solved) atomicAdd(&p.stats[ST_ELBM_SOLVED], (unsigned long long)solved);
        if (skipped) atomicAdd(&p.stats[ST_ELBM_SKIPPED], (unsigned long long)skipped);
        if (fallback) atomicAdd(&p.stats[ST_ELBM_FALLBACK], (unsigned long long)fallback);
        if (iters) atomicAdd(&p.stats[ST_ELBM_ITERS], (unsigned long long)iters);
        if (itmax) atomicMax(&p.stats[ST_ELBM_ITERS_MAX], (unsigned long long)itmax);
    }
}

// CTA-wide sums of a and b added to partial-sum slot (linear block id mod
// kRedSlots) of p.red (and, with two, of p.red + kRedSlots).  Every thread
// of the CTA calls it.  The CTA's sum is formed in T (FP32 in the 16/32-bit
// modes: 256 values, relative error ~5e-7 at worst, far below the FP32
// parity bound) by two shuffle stages, and one FP64 atomic per CTA adds it:
// GB300's narrow FP64 pipe would otherwise hold every CTA at its end.
template <class T>
__device__ __forceinline__ void block_sum_to_slots(const Params& p, T a, T b, bool two) {
    __shared__ T red_a[32], red_b[32];
    const unsigned full = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(full, a, o);
        if (two) b += __shfl_xor_sync(full, b, o);
    }
    const int t = threadIdx.y * blockDim.x + threadIdx.x, w = t >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    if ((t & 31) == 0) {
        red_a[w] = a;
        red_b[w] = b;
    }
    __syncthreads();
    if (t < 32) {
        a = t < nw ? red_a[t] : T(0);
        b = (two && t < nw) ? red_b[t] : T(0);
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(full, a, o);
            if (two) b += __shfl_xor_sync(full, b, o);
        }
        if (t == 0) {
            const unsigned slot = (blockIdx.y * gridDim.x + blockIdx.x) & (kRedSlots - 1);
            if (a != T(0)) atomicAdd(&p.red[slot], (double)a);
            if (two && b != T(0)) atomicAdd(&p.red[kRedSlots + slot], (double)b);
        }
    }
}

// Resident 256-thread CTAs per SM the FP32-arithmetic step kernels are
// compiled for: the streaming step needs the warps to hide HBM latency.
// Ehrenfest and positivity: eight (32 registers, a few bytes of spills;
// measured 4% faster than six); median: six (at 32 registers its FP32
// Delta S spills ~200 bytes) and the Section 4.2-4.4 limiters (four bytes
// of spills).  0 leaves the choice to the compiler (LBGK and
// MRT fit in 32-38 registers by themselves; ELBM and FP64 storage are not
// capped).
template <class ST, int COLL>
constexpr int kMinBlocks =
    (COLL == LBM_ELBM && sizeof(typename ST::T) == 8)
        ? 2  // 128 registers: two CTAs per SM also near rest, where the step streams
        : sizeof(typename ST::T) != 4
        ? 0
        : (COLL == LBM_EHRENFEST || COLL == LBM_POSITIVITY || COLL == LBM_MRT_LIMITER)
              ? 8
              : (COLL == LBM_MEDIAN || (COLL >= LBM_SMOOTH && COLL <= LBM_THRESHOLD) || COLL == LBM_ENSEMBLE_LAGGED)
                    ? 6
                    : 0;

// L2 prefetch of the rows (and the row on either side, for the odd step's
// shifted reads) of the tile that the CTA one resident wave later processes
// (tiles of tw sites x blockDim.y rows in a 2D grid, ctas_per_sm resident
// CTAs per SM): one bulk prefetch per plane row by the CTA's first threads,
// so that the DRAM reads of that tile are under way before it starts.  Only
// on padded layouts (pitch and planes multiples of 32 elements, a 256-byte
// aligned base): every segment then starts on a tile boundary, 16-byte
// aligned, and ends within the padded row with a multiple of 16 bytes; a
// caller's dense array may be neither.
template <int Q, class ST>
__device__ __forceinline__ void prefetch_ahead(const Params& p, int tw, int ctas_per_sm) {
    constexpr int b = (int)sizeof(typename ST::S);
    const bool padded = (p.pitch & 31) == 0 && (p.plane32 & 31) == 0 && ((uintptr_t)p.f & 255u) == 0;
    const int ahead = p.pipe_ctas / 8 * ctas_per_sm;  // SMs x resident CTAs
    const int L = blockIdx.y * gridDim.x + blockIdx.x + ahead;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nrow = blockDim.y + 2;
    if (!padded || L >= (int)(gridDim.x * gridDim.y) || t >= Q * nrow) return;
    const int bx = L % gridDim.x, by = L / gridDim.x;
    const int tx0 = bx * tw, pl = t / nrow, yy = by * blockDim.y - 1 + (t - pl * nrow);
    const int room = p.pitch - tx0;  // a multiple of 32 elements
    const int n = room < tw ? room : tw;
    if (yy < 0 || yy >= p.ny || n <= 0) return;
    const char* a = reinterpret_cast<const char*>(p.f) + ((int64_t)pl * p.plane32 + (int64_t)yy * p.pitch + tx0) * b;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(n * b)) : "memory");
}

// The one-site kernel prefetches the next wave's tiles (prefetch_ahead) in
// FP32 storage for the collisions it speeds up (measured, 4097^2: LBGK
// 0.963 -> 1.02 of the measured copy bandwidth, Ehrenfest 0.948 -> 0.975,
// median 0.930 -> 0.956, positivity, MRT and A_2 to 1.00-1.02, MRT limiter
// 0.954 -> 0.982, smooth limiter 0.857 -> 0.907); the lagged-ensemble and
// threshold steps, which end in a CTA-wide reduction, ran 9-11% slower with it.
template <int Q, class ST, int COLL>
constexpr bool kSitePrefetch = Q == 9 && sizeof(typename ST::S) == 4 &&
                               (COLL == LBM_LBGK || COLL == LBM_EHRENFEST || COLL == LBM_MEDIAN ||
                                COLL == LBM_POSITIVITY || COLL == LBM_MRT || COLL == LBM_MRT2 ||
                                COLL == LBM_MRT_LIMITER || COLL == LBM_SMOOTH);

template <int Q, class ST, int COLL, bool ODD>
__global__ void __launch_bounds__(kBlockX* kBlockY, kMinBlocks<ST, COLL>) step_kernel(Params p) {
    pdl_enter();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    constexpr bool kLimiter =
        (COLL == LBM_EHRENFEST || COLL == LBM_MEDIAN || COLL == LBM_THRESHOLD || COLL == LBM_MRT_LIMITER);
    if (kLimiter && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        p.counters[p.cslot ^ 1] = 0u;  // the next step's list starts empty
        p.counters[CNT_NVALID] = 0u;   // counted by this step's eval / median kernel
    }
    if (kSitePrefetch<Q, ST, COLL>) prefetch_ahead<Q, ST>(p, kBlockX, 8);
    int e_code = -1, e_iters = 0;
    typename ST::T acc = 0;
    if (x < p.nx && y < p.ny) site_update<Q, ST, COLL, ODD>(p, x, y, e_code, e_iters, acc);
    if (COLL == LBM_ELBM) elbm_stats(p, e_code, e_iters);
    if (COLL == LBM_THRESHOLD) block_sum_to_slots<typename ST::T>(p, acc, 0, false);
    if (COLL == LBM_ENSEMBLE_LAGGED)
        block_sum_to_slots<typename ST::T>(p, acc, e_code == 1 ? typename ST::T(1) : typename ST::T(0), true);
}

// Two sites per thread (x0 = 2t, x0 + 1): every population plane moves with
// one aligned 32-bit access per thread holding the pair (and one packed
// conversion).  In odd steps the planes with v_x = +-1 are one element off;
// their two elements are read and written as two 16-bit accesses (a warp's
// 16-bit accesses still cover one contiguous 128-byte row segment).  That
// costs fewer instructions than assembling the shifted pair from the packed
// words of neighbouring lanes (a shuffle and a byte permute per plane and
// direction, conditional accesses at the warp edges): 8-9% faster on the
// screened collisions, 3% on LBGK.  Each element is written only by the
// thread of the site that owns it.  Warps that touch a wall, the domain edge
// or a ragged end take the per-site path.
// The collision runs on both sites at once with the packed FP32 pair
// instructions (collide_dev<F2>).  Used for the 16-bit formats, whose
// per-site instruction count (conversions, addressing) otherwise limits
// them below the HBM roofline; with FP32 storage the one-site kernel is as
// fast or faster.  Compiled for five resident CTAs (48 registers; the
// register pairs of the packed form need more than the one-site form's 40).
constexpr int kVecX = 64;
constexpr int kVecY = 4;
template <class ST, int COLL>
constexpr bool kPairedSites = kDeviationForm<9, ST, COLL>;
constexpr int kPairedMinBlocks = 5;
// The L2 prefetch of the next wave's tiles (below) for the collisions it
// speeds up (measured, 4097^2 FP16: LBGK 0.795 -> 0.832 of HBM, A_2 0.797 ->
// 0.823, positivity 0.739 -> 0.753); the screened collisions and MRT, which
// spend more issue slots per site, ran 5-8% slower with it.
template <int COLL>
constexpr bool kPairPrefetch = COLL == LBM_LBGK || COLL == LBM_MRT2 || COLL == LBM_POSITIVITY;

__device__ __forceinline__ uint32_t ld_word(const void* base, int off) {
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint16_t*>(base) + off);
}
__device__ __forceinline__ void st_word(void* base, int off, uint32_t v) {
    *reinterpret_cast<uint32_t*>(reinterpret_cast<uint16_t*>(base) + off) = v;
}

// Both sites of a pair through the one-site step (out of line: the call is
// rare and nothing of the pair's collision is live across it).
template <int Q, class ST, int COLL, bool ODD>
__device__ __noinline__ void pair_again(const Params& p, int x0, int y) {
    int e_code = -1, e_iters = 0;
    typename ST::T acc = 0;
    site_update<Q, ST, COLL, ODD>(p, x0, y, e_code, e_iters, acc);
    site_update<Q, ST, COLL, ODD>(p, x0 + 1, y, e_code, e_iters, acc);
}

template <int Q, class ST, int COLL, bool ODD>
__global__ void __launch_bounds__(kVecX* kVecY, kPairedMinBlocks) step_kernel_v2(Params p) {
    pdl_enter();
    using T = typename ST::T;
    using L = Lat<Q>;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    constexpr bool kLimiter =
        (COLL == LBM_EHRENFEST || COLL == LBM_MEDIAN || COLL == LBM_THRESHOLD || COLL == LBM_MRT_LIMITER);
    if (kLimiter && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        p.counters[p.cslot ^ 1] = 0u;
        p.counters[CNT_NVALID] = 0u;
    }
    if (kPairPrefetch<COLL>) prefetch_ahead<Q, ST>(p, 2 * kVecX, kPairedMinBlocks);
    int e_code = -1, e_iters = 0;
    const unsigned full = 0xffffffffu;
    const bool inner = y > 0 && y < p.ny - 1 && x0 > 0 && x0 + 2 < p.nx;
    if (!__all_sync(full, inner)) {
        if (y < p.ny) {
            T acc = 0;  // no reduction in the collisions of this kernel
            if (x0 < p.nx) site_update<Q, ST, COLL, ODD>(p, x0, y, e_code, e_iters, acc);
            if (x0 + 1 < p.nx) site_update<Q, ST, COLL, ODD>(p, x0 + 1, y, e_code, e_iters, acc);
        }
        return;
    }
    const int o = y * p.pitch + x0;  // even: every word access is 4-byte aligned
    void* base = p.f;
    using S = typename ST::S;
    // the pairs of the planes read at the site's own column (all planes in
    // even steps) are aligned words; in odd steps the planes with v_x = +-1
    // are one element off, read as two 16-bit loads (sources x0 - v_x and
    // x0 + 1 - v_x).  Every load is issued before any is used.
    uint32_t W[Q];
    S A[Q], B[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int k = ODD ? L::opp(i) : i;
        const int off = k * p.plane32 + o - (ODD ? L::cy(i) * p.pitch : 0);
        if (!ODD || L::cx(i) == 0) {
            W[i] = ld_word(base, off);  // elements x0, x0 + 1 of the plane row
        } else {
            A[i] = reinterpret_cast<const S*>(base)[off - L::cx(i)];
            B[i] = reinterpret_cast<const S*>(base)[off + 1 - L::cx(i)];
        }
    }
    F2 dv[Q];  // deviations f - W of the two sites
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (!ODD || L::cx(i) == 0) {
            const float2 v = ST::unpack(W[i]);
            dv[i] = vmake<F2>(v.x, v.y);
        } else {
            dv[i] = vmake<F2>(ST::dec(A[i]), ST::dec(B[i]));
        }
    }
    F2 Dv[Q];  // post-collision deviations F - W of both sites
    unsigned scr = 0u;
    collide_dev<F2, ST, COLL>(p, x0, y, dv, Dv, &scr);
    if (scr) {
        // a screened site (rare): nothing is stored yet, so both sites run
        // again from the unchanged state through the one-site form, which
        // records the candidate
        pair_again<Q, ST, COLL, ODD>(p, x0, y);
        return;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int k = ODD ? L::opp(i) : i;
        const int off = k * p.plane32 + o - (ODD ? L::cy(i) * p.pitch : 0);
        const float Fa = vlane(Dv[L::opp(i)], 0), Fb = vlane(Dv[L::opp(i)], 1);
        if (!ODD || L::cx(i) == 0) {
            st_word(base, off, ST::pack(Fa, Fb));
        } else {  // a -> x0 - v_x, b -> x0 + 1 - v_x
            reinterpret_cast<S*>(base)[off - L::cx(i)] = ST::enc(Fa);
            reinterpret_cast<S*>(base)[off + 1 - L::cx(i)] = ST::enc(Fb);
        }
    }
}

// Writes F for a candidate site recorded by the step kernel (same parity).
template <int Q, class ST, bool ODD>
__device__ __forceinline__ void rewrite_site(const Params& p, int site, const typename ST::T* F) {
    store_general<Q, ST, ODD>(p, site % p.nx, site / p.nx, F);
}


template <int Q, class ST>
__device__ __forceinline__ void load_candidate(const Params& p, int j, typename ST::T* f) {
    using T = typename ST::T;
    const T* cf = (const T*)p.cand_f;
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = cf[(int64_t)i * p.cand_cap + j];
}

// FP64 Delta S of one site, computed by a group of 16 lanes (lane q < Q
// holds population q in v): the moments and the sum over populations are
// shuffle reductions, so the dependent chain of FP64 operations - the
// latency of this step on GB300's narrow FP64 pipe - is about one
// population's instead of Q.  With inv = 0, v is the pre-collision f; with
// inv = 1 / (1 - 2 beta), v is the post-collision state of an LBGK site, and
// the pre-collision f = f* + (v - f*) inv (LBGK keeps rho and u, so f* is
// the same).  All 32 lanes of the warp must call it (the series length of
// g is chosen once per warp, so that the lanes take one branch: the
// longest any lane needs); inactive lanes (valid = false, or q >= Q)
// contribute nothing.
template <int Q>
__device__ __forceinline__ double delta_s_lanes(const Params& p, double v, bool valid, double inv) {
    const int q = threadIdx.x & 15;
    const unsigned gmask = 0xffffu << (threadIdx.x & 16);
    const bool act = valid && q < Q;
    const int cx = Q == 3 ? q - 1 : ((q == 1 || q == 2 || q == 8) ? 1 : ((q == 4 || q == 5 || q == 6) ? -1 : 0));
    const int cy = Q == 3 ? 0 : ((q == 6 || q == 7 || q == 8) ? 1 : ((q == 2 || q == 3 || q == 4) ? -1 : 0));
    if (!act) v = 0.0;
    double r = v, jx = cx * v, jy = cy * v;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        r += __shfl_xor_sync(gmask, r, o);
        jx += __shfl_xor_sync(gmask, jx, o);
        jy += __shfl_xor_sync(gmask, jy, o);
    }
    double x = 0.0, fe = 0.0;
    bool neg = false;
    if (act) {
        const double ri = 1.0 / r, ux = jx * ri, uy = jy * ri;
        double ax[3], ay[3];
        if (p.eq == LBM_EQ_ENTROPIC) {
            eq1d_entropic<double>(ux, ax[0], ax[1], ax[2]);
            eq1d_entropic<double>(uy, ay[0], ay[1], ay[2]);
        } else {
            eq1d_poly<double>(ux, ax[0], ax[1], ax[2]);
            eq1d_poly<double>(uy, ay[0], ay[1], ay[2]);
        }
        if (Q == 9 && p.eq == LBM_EQ_POLY_STD) {
            // same values as equilibrium<9, double>: the rest population is
            // rho minus the others
            double fi[9], rest = r;
            const double uu = ux * ux + uy * uy;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const double cu = Lat<9>::cx(i) * ux + Lat<9>::cy(i) * uy;
                fi[i] = Lat<9>::w(i) * r * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
                rest -= fi[i];
            }
            fi[0] = rest;
            fe = fi[q];
        } else {
            fe = Q == 3 ? r * ax[cx + 1] : r * ax[cx + 1] * ay[cy + 1];
        }
        const double d = inv != 0.0 ? (v - fe) * inv : v - fe;  // f - f*
        neg = (inv != 0.0 ? fe + d : v) < 0.0 || !(fe > 0.0);
        x = d / fe;
    }
    // one tier of gfun_d for the warp: the series (or log) its largest |x| needs
    const float axf = fminf((float)fabs(x), 2.0f);
    const float am = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(axf)));
    double g;
    if (am < 0.015625f) g = gseries_d<8>(x);
    else if (am < 0.125f) g = gseries_d<16>(x);
    else if (am < 0.25f) g = gseries_d<26>(x);
    else g = x <= -1.0 ? 1.0 : (1.0 + x) * log1p(x) - x;
    double term = act ? fe * g : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) term += __shfl_xor_sync(gmask, term, o);
    neg = __any_sync(gmask, neg);
    return neg ? __longlong_as_double(0x7ff0000000000000ULL) : term;
}

// FP64 Delta S of candidate record j (its recorded pre-collision
// populations); lanes of a group with j >= M pass valid = false and get 0.
template <int Q, class ST>
__device__ __forceinline__ double delta_s_group(const Params& p, unsigned j, bool valid) {
    using T = typename ST::T;
    const int q = threadIdx.x & 15;
    double f = 0.0;
    if (valid && q < Q) f = (double)((const T*)p.cand_f)[(int64_t)q * p.cand_cap + j];
    return delta_s_lanes<Q>(p, f, valid, 0.0);
}

// Ehrenfest regularisation (Section 4): the k candidates with the largest
// Delta S (ties: lower site index) jump to f*.  One CTA; Delta S > delta >= 0
// so the IEEE bit patterns order like the values (+inf last).
// One radix digit of the selection, by the first warp: the digit d whose bin
// holds the rem-th key counting from the top (descending) or from the bottom
// (ascending); rem becomes the rank inside that bin.  Lane l owns eight
// consecutive bins in scan order; a shuffle prefix sum finds the lane.
__device__ __forceinline__ int pick_digit(const unsigned* hist, unsigned& rem, bool descending) {
    const int l = threadIdx.x & 31;
    unsigned c = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) c += hist[descending ? 255 - 8 * l - k : 8 * l + k];
    unsigned incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
        if (l >= off) incl += v;
    }
    const unsigned hit = __ballot_sync(0xffffffffu, incl >= rem);
    const int L = hit ? __ffs(hit) - 1 : 31;
    int digit = 0;
    unsigned r = 0;
    if (l == L) {
        r = rem - (incl - c);
        int k = 0;
        for (; k < 7; ++k) {
            const unsigned h = hist[descending ? 255 - 8 * l - k : 8 * l + k];
            if (h >= r) break;
            r -= h;
        }
        digit = descending ? 255 - 8 * l - k : 8 * l + k;
    }
    digit = __shfl_sync(0xffffffffu, digit, L);
    rem = __shfl_sync(0xffffffffu, r, L);
    return digit;
}

// Sum over the CTA, returned to every thread (every thread calls it).
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double part[32];
    __shared__ double total;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();  // part / total free from a previous call
    if ((t & 31) == 0) part[t >> 5] = v;
    __syncthreads();
    if (t < 32) {
        double u = t < nw ? part[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
        if (t == 0) total = u;
    }
    __syncthreads();
    return total;
}

// Threshold limiter (Section 4.4), one CTA after every cand_ds entry of the
// step is final (FP64 Delta S of the screened sites, -1 where not above
// delta).  With S the step's sum of Delta S over the lattice (partial sums
// of the step kernel) and R = delta0 (1 - (2 beta - 1)^2) S, the threshold
// Delta S_0 of Eq. (EntThresh) solves L(t) = sum max(Delta S - t, 0) = R.
// Only sites above delta matter when L(delta) > R (otherwise Delta S_t =
// delta); then the sites whose L(Delta S) < R (the "upper" set, n of them
// with sum S_u) are found by an MSB radix descent over the FP64 bits of the
// candidate values with per-bin counts and sums, and Delta S_0 =
// (S_u - R) / n, the root on the linear piece of L below them.  Sites with
// Delta S >= Delta S_t = max(Delta S_0, delta) get the homothety
// sqrt(Delta S_t / Delta S) of Eq. (entrHom) before the LBGK collision.
template <int Q, class ST, bool ODD>
__device__ void threshold_select_apply(const Params& p, unsigned M) {
    using T = typename ST::T;
    __shared__ unsigned cnt[256];
    __shared__ double hsum[256];
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ double s_cntA, s_sumA;
    __shared__ int s_done;
    __shared__ unsigned s_count;
    const int tid = threadIdx.x, nt = blockDim.x;
    // the step's sum of Delta S; the slots are cleared for the next step
    double S = 0.0;
    for (int k = tid; k < kRedSlots; k += nt) {
        S += __ldcg(&p.red[k]);
        p.red[k] = 0.0;
    }
    S = block_sum(S);
    const double c = 1.0 - (2.0 * p.beta - 1.0) * (2.0 * p.beta - 1.0);
    const double R = p.lim_delta0 * c * S;
    double Ld = 0.0;
    for (unsigned j = tid; j < M; j += nt) {
        const double v = __ldcg(&p.cand_ds[j]);
        if (v > p.delta && v < INFINITY) Ld += v - p.delta;
    }
    Ld = block_sum(Ld);
    double dst = p.delta;
    if (Ld > R) {
        if (tid == 0) {
            s_prefix = 0ull;
            s_mask = 0ull;
            s_cntA = 0.0;
            s_sumA = 0.0;
            s_done = 0;
        }
        __syncthreads();
        for (int shift = 56; shift >= 0; shift -= 8) {
            if (s_done) break;  // uniform: read after the barrier
            for (int d = tid; d < 256; d += nt) {
                cnt[d] = 0u;
                hsum[d] = 0.0;
            }
            __syncthreads();
            const unsigned long long pre = s_prefix, msk = s_mask;
            for (unsigned j = tid; j < M; j += nt) {
                const double v = __ldcg(&p.cand_ds[j]);
                if (!(v > p.delta && v < INFINITY)) continue;
                const unsigned long long key = (unsigned long long)__double_as_longlong(v);
                if ((key & msk) != pre) continue;
                const int d = (int)((key >> shift) & 255ull);
                atomicAdd(&cnt[d], 1u);
                atomicAdd(&hsum[d], v);
            }
            __syncthreads();
            if (tid == 0) {
                // bins from the top: the first whose lower bound b has
                // L(b) >= R holds the boundary; the bins above it are upper
                double cA = s_cntA, sA = s_sumA;
                int chosen = -1;
                for (int d = 255; d >= 0; --d) {
                    const double ci = cA + (double)cnt[d], si = sA + hsum[d];
                    const double b = __longlong_as_double((long long)(pre | ((unsigned long long)d << shift)));
                    if (si - b * ci >= R) {
                        chosen = d;
                        break;
                    }
                    cA = ci;
                    sA = si;
                }
                s_cntA = cA;
                s_sumA = sA;
                if (chosen < 0) {
                    s_done = 1;
                } else {
                    s_prefix = pre | ((unsigned long long)chosen << shift);
                    s_mask = msk | (255ull << shift);
                }
            }
            __syncthreads();
        }
        // n = 0: R <= 0 and the boundary is the largest value itself
        const double t0 = s_cntA > 0.0 ? (s_sumA - R) / s_cntA : __longlong_as_double((long long)s_prefix);
        dst = t0 > p.delta ? t0 : p.delta;
    }
    if (tid == 0) s_count = 0u;
    __syncthreads();
    unsigned mine = 0;
    const T om1 = sizeof(T) == 8 ? T(1.0 - 2.0 * p.beta) : T(1) - T(2) * T(p.beta_f);
    for (unsigned j = tid; j < M; j += nt) {
        const double v = __ldcg(&p.cand_ds[j]);
        const bool sel = v >= dst;  // +inf included, -1 (not above delta) excluded
        p.cand_sel[j] = sel ? 1 : 0;
        if (!sel) continue;
        const T phi = v < INFINITY ? T(sqrt(dst / v)) : T(0);
        T f[Q], feq[Q], F[Q], rho, ux, uy;
        load_candidate<Q, ST>(p, (int)j, f);
        moments<Q, T>(f, rho, ux, uy);
        equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
#pragma unroll
        for (int i = 0; i < Q; ++i) F[i] = feq[i] + om1 * phi * (f[i] - feq[i]);
        conserve_mass<Q, T>(rho, F);
        rewrite_site<Q, ST, ODD>(p, p.cand_site[j], F);
        ++mine;
    }
    if (mine) atomicAdd(&s_count, mine);
    __syncthreads();
    if (tid == 0) {
        p.counters[CNT_NSEL] = s_count;
        if (s_count) atomicAdd(&p.stats[ST_LIMITED], (unsigned long long)s_count);
        *p.lim_E = dst;  // the step's Delta S_t, for inspection
    }
}

// Runs in one CTA of any size after every cand_ds entry of the step is final
// (the entries of other CTAs are read through L2).
template <int Q, class ST, bool ODD, int COLL = LBM_EHRENFEST>
__device__ void ehrenfest_select_apply(const Params& p, unsigned M, unsigned nvalid) {
    using T = typename ST::T;
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix, s_mask;
    __shared__ unsigned s_rem;
    __shared__ unsigned s_count;
    __shared__ int s_ties_all;
    const int tid = threadIdx.x;
    const unsigned K = p.topk > 0 ? (unsigned)p.topk : 0u;
    // candidates: screened sites whose FP64 Delta S exceeds delta (the others
    // carry -1); their keys are positive doubles.  Up to kCache per thread
    // are held in registers across the radix passes (else re-read per pass).
    constexpr int kCache = 4;
    const bool cached = M <= kCache * blockDim.x;
    double kds[kCache];
    unsigned ksite[kCache];
#pragma unroll
    for (int i = 0; i < kCache; ++i) {
        const unsigned j = tid + i * blockDim.x;
        const bool in = cached && j < M;
        kds[i] = in ? __ldcg(&p.cand_ds[j]) : -1.0;
        ksite[i] = in ? (unsigned)__ldcg(&p.cand_site[j]) : 0u;
    }
    // visits (ds, site) of every record this thread owns
    auto each = [&](auto&& fn) {
        if (cached) {
#pragma unroll
            for (int i = 0; i < kCache; ++i) {
                const unsigned j = tid + i * blockDim.x;
                if (j < M) fn(j, kds[i], ksite[i]);
            }
        } else {
            for (unsigned j = tid; j < M; j += blockDim.x)
                fn(j, __ldcg(&p.cand_ds[j]), (unsigned)__ldcg(&p.cand_site[j]));
        }
    };
    if (tid == 0) s_count = 0;
    const bool all = nvalid <= K;
    unsigned long long tkey = 0;
    unsigned icut = 0xffffffffu;
    if (!all && K > 0) {
        // MSB-first radix select of the K-th largest key, 8 bits per pass
        if (tid == 0) {
            s_prefix = 0;
            s_mask = 0;
            s_rem = K;
            s_ties_all = 0;
        }
        __syncthreads();
        for (int shift = 56; shift >= 0; shift -= 8) {
            for (int d = tid; d < 256; d += blockDim.x) hist[d] = 0;
            __syncthreads();
            const unsigned long long pre = s_prefix, msk = s_mask;
            each([&](unsigned, double ds, unsigned) {
                const unsigned long long key = (unsigned long long)__double_as_longlong(ds);
                if (ds > p.delta && (key & msk) == pre) atomicAdd(&hist[(key >> shift) & 255ull], 1u);
            });
            __syncthreads();
            if (tid < 32) {
                unsigned rem = s_rem;
                const int d = pick_digit(hist, rem, true);
                if (tid == 0) {
                    s_rem = rem;
                    s_prefix = pre | ((unsigned long long)d << shift);
                    s_mask = msk | (255ull << shift);
                    // the last bin holds the keys equal to the K-th: all taken?
                    if (shift == 0) s_ties_all = hist[d] == rem;
                }
            }
            __syncthreads();
        }
        tkey = s_prefix;
        const bool ties_all = s_ties_all;
        __syncthreads();  // every thread has read the threshold before it is reused
        if (!ties_all) {
            // among keys equal to the threshold, take the s_rem smallest sites
            if (tid == 0) {
                s_prefix = 0;
                s_mask = 0;
            }
            __syncthreads();
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int d = tid; d < 256; d += blockDim.x) hist[d] = 0;
                __syncthreads();
                const unsigned pre = (unsigned)s_prefix, msk = (unsigned)s_mask;
                each([&](unsigned, double ds, unsigned site) {
                    const unsigned long long key = (unsigned long long)__double_as_longlong(ds);
                    if (ds > p.delta && key == tkey && (site & msk) == pre)
                        atomicAdd(&hist[(site >> shift) & 255u], 1u);
                });
                __syncthreads();
                if (tid < 32) {
                    unsigned rem = s_rem;
                    const int d = pick_digit(hist, rem, false);
                    if (tid == 0) {
                        s_rem = rem;
                        s_prefix = pre | ((unsigned)d << shift);
                        s_mask = msk | (255u << shift);
                    }
                }
                __syncthreads();
            }
            icut = (unsigned)s_prefix;
        }
    }
    __syncthreads();
    unsigned mine = 0;
    each([&](unsigned j, double ds, unsigned site) {
        bool sel = false;
        if (K > 0 && ds > p.delta) {
            if (all) {
                sel = true;
            } else {
                const unsigned long long key = (unsigned long long)__double_as_longlong(ds);
                sel = key > tkey || (key == tkey && site <= icut);
            }
        }
        p.cand_sel[j] = sel ? 1 : 0;
        if (sel) {
            T f[Q], feq[Q], rho, ux, uy;
            load_candidate<Q, ST>(p, (int)j, f);
            moments<Q, T>(f, rho, ux, uy);
            equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
            if constexpr (COLL == LBM_MRT_LIMITER && Q == 9) {
                // Section 5's MRT limiter: the selected site takes A_2, not f*
                T F[Q];
                mrt2_d2q9<T>(f, feq, sizeof(T) == 8 ? T(2.0 * p.beta) : T(2) * T(p.beta_f), F);
                conserve_mass<Q, T>(rho, F);
                rewrite_site<Q, ST, ODD>(p, (int)site, F);
            } else {
                conserve_mass<Q, T>(rho, feq);
                rewrite_site<Q, ST, ODD>(p, (int)site, feq);
            }
            ++mine;
        }
    });
    if (mine) atomicAdd(&s_count, mine);
    __syncthreads();
    if (tid == 0) {
        p.counters[CNT_NSEL] = s_count;
        if (s_count) atomicAdd(&p.stats[ST_LIMITED], (unsigned long long)s_count);
    }
}

// Ehrenfest step, second kernel: the FP64 Delta S of every screened site
// (grid-stride), then the last CTA to finish - found by a ticket counter after
// a memory fence, no waiting - selects the k largest and rewrites them.
template <int Q, class ST, bool ODD, int COLL>
__device__ __forceinline__ void select_apply(const Params& p, unsigned M, unsigned nvalid) {
    if constexpr (COLL == LBM_THRESHOLD)
        threshold_select_apply<Q, ST, ODD>(p, M);
    else
        ehrenfest_select_apply<Q, ST, ODD, COLL>(p, M, nvalid);
}

// The post-collision state of selected record j written back (f*, or A_2
// for the MRT limiter).
template <int Q, class ST, int COLL, bool ODD>
__device__ __forceinline__ void rewrite_selected(const Params& p, unsigned j) {
    using T = typename ST::T;
    T f[Q], feq[Q], rho, ux, uy;
    load_candidate<Q, ST>(p, (int)j, f);
    moments<Q, T>(f, rho, ux, uy);
    equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
    const int site = p.cand_site[j];
    if constexpr (COLL == LBM_MRT_LIMITER && Q == 9) {
        T F[Q];
        mrt2_d2q9<T>(f, feq, sizeof(T) == 8 ? T(2.0 * p.beta) : T(2) * T(p.beta_f), F);
        conserve_mass<Q, T>(rho, F);
        rewrite_site<Q, ST, ODD>(p, site, F);
    } else {
        conserve_mass<Q, T>(rho, feq);
        rewrite_site<Q, ST, ODD>(p, site, feq);
    }
}

constexpr int64_t kSettleSites = 1 << 21;

// Up to two screened records per thread: every CTA settles every record's
// side of delta in FP32 (certify_side; the same result in each CTA).  When
// every side is settled and at most k records are above delta, the first
// CTA takes all of those without FP64 work and the call returns true in
// every CTA; otherwise it returns false everywhere and the grid-wide FP64
// evaluation decides.  Out of line: inlined, its code in front of the other
// paths slowed the selection kernel of large lattices (measured).
template <int Q, class ST, bool ODD, int COLL>
__device__ __noinline__ bool settle_all_taken(const Params& p, unsigned M) {
    using T = typename ST::T;
    const unsigned tid = threadIdx.x, nt = blockDim.x;
    int side[2];
    float ds32[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const unsigned j = tid + r * nt;
        side[r] = 0;
        ds32[r] = 0.f;
        if (j < M) {
            T f[Q];
            float ff[Q];
            load_candidate<Q, ST>(p, (int)j, f);
#pragma unroll
            for (int i = 0; i < Q; ++i) ff[i] = (float)f[i];
            side[r] = certify_side<Q>(p, ff, ds32[r]);
        }
    }
    const int unsure = __syncthreads_or(side[0] == 2 || side[1] == 2);
    const unsigned nabove = (unsigned)__syncthreads_count(side[0] == 1) + (unsigned)__syncthreads_count(side[1] == 1);
    const unsigned K = p.topk > 0 ? (unsigned)p.topk : 0u;
    if (unsure || nabove > K) return false;
    if (blockIdx.x != 0) return true;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const unsigned j = tid + r * nt;
        if (j >= M) continue;
        const bool sel = side[r] == 1;
        p.cand_sel[j] = sel ? 1 : 0;
        p.cand_ds[j] = sel ? (double)ds32[r] : -1.0;  // lbm_last_candidates recomputes FP64 values
        if (sel) rewrite_selected<Q, ST, COLL, ODD>(p, j);
    }
    if (tid == 0) {
        p.counters[CNT_NVALID] = nabove;
        p.counters[CNT_NSEL] = nabove;
        if (nabove) atomicAdd(&p.stats[ST_LIMITED], (unsigned long long)nabove);
    }
    return true;
}

template <int Q, class ST, bool ODD, int COLL>
__device__ __forceinline__ void eval_then_select(const Params& p) {
    __shared__ unsigned s_last;
    unsigned M = p.counters[p.cslot];
    if (M > (unsigned)p.cand_cap) M = (unsigned)p.cand_cap;
    if constexpr (COLL != LBM_THRESHOLD) {
        // small lattices only: there the selection's latency is most of the
        // step, while on large ones the grid-wide pass hides under the next
        // step's launch and a failed attempt would only add to it (measured)
        if ((int64_t)p.nx * p.ny <= kSettleSites && M > (blockDim.x >> 4) && M <= 2 * blockDim.x &&
            settle_all_taken<Q, ST, ODD, COLL>(p, M))
            return;
    }
    if (M <= (blockDim.x >> 4)) {
        // few screened sites (the usual case): the first CTA evaluates them
        // all, one 16-lane group each, and selects without the ticket and
        // its memory fences; the other CTAs have nothing to do
        if (blockIdx.x != 0) return;
        __shared__ double s_key[16];
        __shared__ int s_site[16];
        __shared__ unsigned s_nsel;
        const unsigned j = threadIdx.x >> 4;
        const bool lead = j < M && (threadIdx.x & 15) == 0;
        if (threadIdx.x == 0) {
            s_last = 0;
            s_nsel = 0;
        }
        if constexpr (COLL != LBM_THRESHOLD) {
            // every screened site certainly on one side of delta in FP32 and
            // no more candidates than k: all of them are taken, no FP64
            // Delta S (FP64 storage: the records rounded to FP32 move Delta S
            // by at most 6e-8 sqrt(q rho), inside the same bound)
            using T = typename ST::T;
            T f[Q];
            float ds32 = 0.f;
            int side = 0;
            if (lead) {
                load_candidate<Q, ST>(p, (int)j, f);
                float ff[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) ff[i] = (float)f[i];
                side = certify_side<Q>(p, ff, ds32);
            }
            const int unsure = __syncthreads_or(lead && side == 2);
            const unsigned ncert = (unsigned)__syncthreads_count(lead && side == 1);
            const unsigned K = p.topk > 0 ? (unsigned)p.topk : 0u;
            if (!unsure && ncert <= K) {
                if (lead) {
                    const bool sel = side == 1;
                    p.cand_sel[j] = sel ? 1 : 0;
                    // the FP32 value of a selected site (lbm_last_candidates
                    // recomputes FP64 values)
                    p.cand_ds[j] = sel ? (double)ds32 : -1.0;
                    if (sel) {
                        T feq[Q], rho, ux, uy;
                        moments<Q, T>(f, rho, ux, uy);
                        equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
                        const int site = p.cand_site[j];
                        if constexpr (COLL == LBM_MRT_LIMITER && Q == 9) {
                            T F[Q];
                            mrt2_d2q9<T>(f, feq, sizeof(T) == 8 ? T(2.0 * p.beta) : T(2) * T(p.beta_f), F);
                            conserve_mass<Q, T>(rho, F);
                            rewrite_site<Q, ST, ODD>(p, site, F);
                        } else {
                            conserve_mass<Q, T>(rho, feq);
                            rewrite_site<Q, ST, ODD>(p, site, feq);
                        }
                    }
                }
                if (threadIdx.x == 0) {
                    p.counters[CNT_NVALID] = ncert;
                    p.counters[CNT_NSEL] = ncert;
                    if (ncert) atomicAdd(&p.stats[ST_LIMITED], (unsigned long long)ncert);
                }
                return;
            }
        }
        __syncthreads();
        const double d = delta_s_group<Q, ST>(p, j, j < M);
        const bool c = lead && d > p.delta;
        int site = 0;
        if (lead) {
            site = p.cand_site[j];
            p.cand_ds[j] = c ? d : -1.0;
            s_key[j] = c ? d : -1.0;
            s_site[j] = site;
            if (c) atomicAdd(&s_last, 1u);
        }
        __syncthreads();  // this CTA's cand_ds entries are final
        const unsigned nvalid = s_last;
        if (threadIdx.x == 0) p.counters[CNT_NVALID] = nvalid;
        if constexpr (COLL == LBM_THRESHOLD) {
            select_apply<Q, ST, ODD, COLL>(p, M, nvalid);
        } else {
            // the k largest: a candidate's rank is the number of candidates
            // before it in (Delta S descending, site ascending) order
            if (lead) {
                const unsigned K = p.topk > 0 ? (unsigned)p.topk : 0u;
                bool sel = false;
                if (c && K > 0) {
                    unsigned rank = 0;
                    for (unsigned i = 0; i < M; ++i) {
                        const double o = s_key[i];
                        rank += (o > d || (o == d && s_site[i] < site)) ? 1u : 0u;
                    }
                    sel = rank < K;
                }
                p.cand_sel[j] = sel ? 1 : 0;
                if (sel) {
                    using T = typename ST::T;
                    T f[Q], feq[Q], rho, ux, uy;
                    load_candidate<Q, ST>(p, (int)j, f);
                    moments<Q, T>(f, rho, ux, uy);
                    equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
                    if constexpr (COLL == LBM_MRT_LIMITER && Q == 9) {
                        T F[Q];
                        mrt2_d2q9<T>(f, feq, sizeof(T) == 8 ? T(2.0 * p.beta) : T(2) * T(p.beta_f), F);
                        conserve_mass<Q, T>(rho, F);
                        rewrite_site<Q, ST, ODD>(p, site, F);
                    } else {
                        conserve_mass<Q, T>(rho, feq);
                        rewrite_site<Q, ST, ODD>(p, site, feq);
                    }
                    atomicAdd(&s_nsel, 1u);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                p.counters[CNT_NSEL] = s_nsel;
                if (s_nsel) atomicAdd(&p.stats[ST_LIMITED], (unsigned long long)s_nsel);
            }
        }
        return;
    }
    unsigned n = 0;
    // one record per 16-lane group
    const unsigned groups = gridDim.x * (blockDim.x >> 4);
    const unsigned g0 = blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4);
    for (unsigned base = 0; base < M; base += groups) {
        const unsigned j = base + g0;
        const double d = delta_s_group<Q, ST>(p, j, j < M);
        if (j < M && (threadIdx.x & 15) == 0) {
            const bool c = d > p.delta;
            p.cand_ds[j] = c ? d : -1.0;
            n += c;
        }
    }
    n = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(&p.counters[CNT_NVALID], n);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&p.counters[CNT_DONE], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const unsigned nvalid = atomicAdd(&p.counters[CNT_NVALID], 0u);
    select_apply<Q, ST, ODD, COLL>(p, M, nvalid);
    if (threadIdx.x == 0) p.counters[CNT_DONE] = 0u;
}

template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256) ehrenfest_eval_select(Params p) {
    pdl_enter();
    eval_then_select<Q, ST, ODD, LBM_EHRENFEST>(p);
}

// MRT limiter (Section 5), second kernel: the Ehrenfest selection; the
// selected sites take the A_2 collision.
template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256) mrt_limiter_eval_select(Params p) {
    pdl_enter();
    eval_then_select<Q, ST, ODD, LBM_MRT_LIMITER>(p);
}

// Threshold limiter, second kernel: FP64 Delta S of the screened sites as
// above, then (one CTA) Delta S_t and the homothety of the sites above it.
template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256) threshold_eval_select(Params p) {
    pdl_enter();
    eval_then_select<Q, ST, ODD, LBM_THRESHOLD>(p);
}

// Lattice mean of the finite Delta S of the pre-collision state of the
// coming step (parity ODD), for the ensemble-dependent limiter: per-CTA sums
// into slots, then the last CTA to finish (ticket after a fence) adds the
// slots, clears them and writes E.
template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256) ensemble_mean(Params p) {
    pdl_enter();
    using T = typename ST::T;
    __shared__ unsigned s_last;
    // a fixed grid strides over row segments of blockDim.x sites (few CTAs:
    // few ticket atomics)
    const int t = threadIdx.x, nt = blockDim.x;
    const int tpr = (p.nx + nt - 1) / nt;
    // tile = y * tpr + seg, advanced by gridDim.x without a division per tile
    const int dy = gridDim.x / tpr, dseg = gridDim.x - dy * tpr;
    int y = blockIdx.x / tpr, seg = blockIdx.x - y * tpr;
    T sum = 0, cnt = 0;
    for (; y < p.ny; y += dy, seg += dseg) {
        if (seg >= tpr) {
            seg -= tpr;
            ++y;
            if (y >= p.ny) break;
        }
        const int x = seg * nt + t;
        if (x >= p.nx) continue;
        T f[Q], feq[Q], rho, ux, uy, q;
        const bool interior = x > 0 && x < p.nx - 1 && (Q == 3 || (y > 0 && y < p.ny - 1));
        if (p.diffusive && !interior) continue;  // wall sites are not in the mean
        if (interior)
            load_interior<Q, ST, ODD>(p, y * p.pitch + x, f);
        else
            load_general<Q, ST, ODD>(p, x, y, f);
        T ds;
        if constexpr (kLimForm<Q, ST, LBM_ENSEMBLE>) {
            // the Delta S the step's collision computes (collide_lim)
            lim_state(p.eq, f, rho, ux, uy, feq);
            ds = delta_s_lim(f, feq, q);
        } else {
            moments<Q, T>(f, rho, ux, uy);
            equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
            ds = delta_s_and_q<Q, T>(f, feq, q);
        }
        if (isfinite(ds)) {
            sum += ds;
            cnt += T(1);
        }
    }
    block_sum_to_slots<T>(p, sum, cnt, true);
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&p.counters[CNT_DONE], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double S = 0.0, N = 0.0;
    for (int k = t; k < kRedSlots; k += nt) {
        S += __ldcg(&p.red[k]);
        N += __ldcg(&p.red[kRedSlots + k]);
        p.red[k] = 0.0;
        p.red[kRedSlots + k] = 0.0;
    }
    S = block_sum(S);
    N = block_sum(N);
    if (t == 0) {
        *p.lim_E = N > 0.0 ? S / N : 0.0;
        *p.lim_E_f = (float)*p.lim_E;
        p.counters[CNT_DONE] = 0u;
    }
}

// Lagged ensemble limiter, after its step: E(Delta S) for the next step from
// the step's partial sums and counts of the finite Delta S (one CTA), the
// slots cleared.
template <class ST>
__global__ void __launch_bounds__(256) ensemble_finalize(Params p) {
    pdl_enter();
    const int t = threadIdx.x;
    double S = 0.0, N = 0.0;
    for (int k = t; k < kRedSlots; k += blockDim.x) {
        S += p.red[k];
        N += p.red[kRedSlots + k];
        p.red[k] = 0.0;
        p.red[kRedSlots + k] = 0.0;
    }
    S = block_sum(S);
    N = block_sum(N);
    if (t == 0) {
        *p.lim_E = N > 0.0 ? S / N : 0.0;
        *p.lim_E_f = (float)*p.lim_E;
    }
}

// Median entropy filter (Section 4.4): lower median of Delta S over the site
// and its neighbours (clipped at walls, wrapped where periodic); where the
// median is below the site's Delta S the homothety with coefficient
// sqrt(med / DeltaS) (Eq. entrHom) precedes the LBGK collision.
// Candidates g0, g0 + G, ... of the step's list, one per 16-lane group
// (g0: this group's index, G: the number of groups; every lane of a group
// calls this).  The FP64 Delta S is the group's; its first lane does the rest.
template <int Q, class ST, bool ODD>
__device__ void median_apply(const Params& p, unsigned g0, unsigned G) {
    using T = typename ST::T;
    unsigned M = p.counters[p.cslot];
    if (M > (unsigned)p.cand_cap) M = (unsigned)p.cand_cap;
    const T* field = (const T*)p.ds_field;
    unsigned count = 0, nvalid = 0;
    for (unsigned b = 0; b < M; b += G) {
        const unsigned j = b + g0;
        const double d = delta_s_group<Q, ST>(p, j, j < M);
        if (j >= M || (threadIdx.x & 15) != 0) continue;
        T f[Q];
        load_candidate<Q, ST>(p, (int)j, f);
        const bool is_cand = d > p.delta;
        p.cand_ds[j] = is_cand ? d : -1.0;
        if (!is_cand) {
            p.cand_sel[j] = 0;
            continue;
        }
        ++nvalid;
        const int site = p.cand_site[j];
        const int x = site % p.nx, y = site / p.nx;
        T w[9];
        int n = 0;
        const int ry = Q == 9 ? 1 : 0;
        // the window is clipped to the fluid sites (all sites except the
        // wall sites of diffusive walls)
        const int lo = p.diffusive ? 1 : 0, hx = p.diffusive ? p.nx - 1 : p.nx, hy = p.diffusive ? p.ny - 1 : p.ny;
        for (int dy = -ry; dy <= ry; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int xx = x + dx, yy = y + dy;
                if (p.periodic_x) xx = xx < 0 ? xx + p.nx : (xx >= p.nx ? xx - p.nx : xx);
                if (p.periodic_y) yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
                if (xx < lo || xx >= hx || yy < (Q == 9 ? lo : 0) || yy >= (Q == 9 ? hy : p.ny)) continue;
                T v = field[(int64_t)yy * p.nx + xx];
                int k = n++;
                while (k > 0 && w[k - 1] > v) {  // insertion sort, ascending
                    w[k] = w[k - 1];
                    --k;
                }
                w[k] = v;
            }
        const T med = w[(n - 1) / 2];
        const T c = field[site];
        const bool sel = med < c;
        p.cand_sel[j] = sel ? 1 : 0;
        if (sel) {
            const T phi = isinf(c) ? T(0) : sqrt(med / c);
            T feq[Q], F[Q], rho, ux, uy;
            moments<Q, T>(f, rho, ux, uy);
            equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
            const T om = T(2) * T(p.beta);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                T fl = feq[i] + phi * (f[i] - feq[i]);
                F[i] = fl + om * (feq[i] - fl);
            }
            conserve_mass<Q, T>(rho, F);
            rewrite_site<Q, ST, ODD>(p, site, F);
            ++count;
        }
    }
    if (count) atomicAdd(&p.stats[ST_LIMITED], (unsigned long long)count);
    if (nvalid) atomicAdd(&p.counters[CNT_NVALID], nvalid);
}

template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256) median_fixup(Params p) {
    pdl_enter();
    median_apply<Q, ST, ODD>(p, blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4), gridDim.x * (blockDim.x >> 4));
}

// Median filter, second kernel, without a Delta S field (|1 - 2 beta| >= 1/16
// for FP32 and FP64 storage, >= 1/4 for 16-bit): the step ran LBGK and the Ehrenfest
// screen at every site, so a window site's pre-collision state is either
// its record (a screened site) or is recovered from its post-collision one
// (delta_s_lanes with inv = 1 / (1 - 2 beta)); its Delta S is FP64.  One
// candidate per CTA and round (one 16-lane group per window site, so the
// narrow FP64 pipe of several SMs shares the work); the first lane of the
// centre group takes the lower median and the new populations.  With at
// most kMedDirect screened sites every window site is looked up in the
// list, no window reads a post-collision state that a rewrite changes, and
// each CTA rewrites its candidate at once; with more, the windows are all
// recovered from the lattice, and the rewrites wait for every window of
// the step: each selected site's coefficient goes to its record and the
// last CTA to finish (ticket after a fence) writes the new populations.
// The post-collision state of median candidate j whose pre-collision state
// gets the homothety with coefficient phi before the LBGK collision.
template <int Q, class ST>
__device__ __forceinline__ void median_homothety(const Params& p, int j, typename ST::T phi, typename ST::T* F) {
    using T = typename ST::T;
    T f[Q], feq[Q], rho, ux, uy;
    load_candidate<Q, ST>(p, j, f);
    moments<Q, T>(f, rho, ux, uy);
    equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
    const T om = T(2) * T(p.beta);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T fl = feq[i] + phi * (f[i] - feq[i]);
        F[i] = fl + om * (feq[i] - fl);
    }
    conserve_mass<Q, T>(rho, F);
}

template <int Q>
struct MedWin {
    static constexpr int W = Q == 9 ? 9 : 3;  // window sites
    static constexpr int centre = W / 2;
};
constexpr unsigned kMedDirect = 64;

template <int Q, class ST, bool ODD>
__global__ void __launch_bounds__(256) median_recon_fixup(Params p) {
    pdl_enter();
    using T = typename ST::T;
    using L = Lat<Q>;
    using MW = MedWin<Q>;
    __shared__ double win[MW::W];
    __shared__ unsigned s_last;
    unsigned M = p.counters[p.cslot];
    if (M > (unsigned)p.cand_cap) M = (unsigned)p.cand_cap;
    const bool direct = M <= kMedDirect;
    const int q = threadIdx.x & 15;
    const unsigned k = threadIdx.x >> 4;  // window site of this group
    const unsigned gmask = 0xffffu << (threadIdx.x & 16);
    // warps without a window site skip the FP64 work (both groups idle)
    const bool warp_works = (threadIdx.x >> 5) * 2 < (unsigned)MW::W;
    const int dx = Q == 9 ? (int)(k % 3) - 1 : (int)k - 1, dy = Q == 9 ? (int)(k / 3) - 1 : 0;
    // the window is clipped to the fluid sites (all sites except the wall
    // sites of diffusive walls)
    const int lo = p.diffusive ? 1 : 0, hx = p.diffusive ? p.nx - 1 : p.nx, hy = p.diffusive ? p.ny - 1 : p.ny;
    const typename ST::S* base = (const typename ST::S*)p.f;
    T* cf = (T*)p.cand_f;
    unsigned nvalid = 0, nsel = 0;
    for (unsigned j = blockIdx.x; j < M; j += gridDim.x) {
        if (warp_works) {
            const bool act = k < (unsigned)MW::W;
            const bool centre = k == (unsigned)MW::centre;
            int xx = 0, yy = 0;
            bool inw = false;
            if (act) {
                const int site = p.cand_site[j];
                xx = site % p.nx + dx;
                yy = site / p.nx + dy;
                if (p.periodic_x) xx = xx < 0 ? xx + p.nx : (xx >= p.nx ? xx - p.nx : xx);
                if (p.periodic_y) yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
                inw = xx >= lo && xx < hx && yy >= (Q == 9 ? lo : 0) && yy < (Q == 9 ? hy : p.ny);
            }
            // the record of the window site, if it has one (direct mode)
            int rec = centre ? (int)j : -1;
            if (direct && act && inw && !centre) {
                const int want = yy * p.nx + xx;
                int found = -1;
                for (unsigned i = q; i < M; i += 16)
                    if (p.cand_site[i] == want) found = (int)i;
                const unsigned hit = __ballot_sync(gmask, found >= 0) & gmask;
                if (hit) rec = __shfl_sync(gmask, found, __ffs(hit) - 1);
            }
            double v = 0.0;
            if (act && inw && q < Q) {
                if (rec >= 0) {
                    v = (double)cf[(int64_t)q * p.cand_cap + rec];
                } else {
                    // population q of the site's post-collision state, where the
                    // step stored it (store_general's addressing, lid term added back)
                    T lidc;
                    const int i = L::opp(q);
                    const int64_t r = aa_address<Q, T>(p, xx, yy, i, ODD, lidc);
                    v = (double)(ST::ld(base + r, T(L::w(i))) + lidc);
                }
            }
            const double ds = delta_s_lanes<Q>(p, v, act && inw, rec >= 0 ? 0.0 : p.median_inv);
            if (q == 0 && act) win[k] = inw ? ds : __longlong_as_double(0x7ff8000000000000LL);
        }
        __syncthreads();
        if (threadIdx.x == 16 * MW::centre) {
            const double c = win[MW::centre];
            const bool cand = c > p.delta;
            p.cand_ds[j] = cand ? c : -1.0;
            bool sel = false;
            if (cand) {
                ++nvalid;
                double w[MW::W];
                int n = 0;
#pragma unroll
                for (int kk = 0; kk < MW::W; ++kk) {
                    const double u = win[kk];
                    if (!(u == u)) continue;  // outside the window
                    int m = n++;
                    while (m > 0 && w[m - 1] > u) {  // insertion sort, ascending
                        w[m] = w[m - 1];
                        --m;
                    }
                    w[m] = u;
                }
                const double med = w[(n - 1) / 2];
                sel = med < c;
                if (sel) {
                    ++nsel;
                    const T phi = isinf(c) ? T(0) : T(sqrt(med / c));
                    if (direct) {
                        T F[Q];
                        median_homothety<Q, ST>(p, (int)j, phi, F);
                        rewrite_site<Q, ST, ODD>(p, p.cand_site[j], F);
                    } else {
                        p.cand_ds[j] = (double)phi;  // for the last CTA (lbm_last_candidates recomputes Delta S)
                    }
                }
            }
            p.cand_sel[j] = sel ? 1 : 0;
        }
        __syncthreads();  // win is reused
    }
    if (threadIdx.x == 16 * MW::centre) {
        if (nvalid) atomicAdd(&p.counters[CNT_NVALID], nvalid);
        if (nsel) atomicAdd(&p.stats[ST_LIMITED], (unsigned long long)nsel);
    }
    if (direct) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&p.counters[CNT_DONE], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (unsigned j = threadIdx.x; j < M; j += blockDim.x) {
        if (!__ldcg(&p.cand_sel[j])) continue;
        T F[Q];
        median_homothety<Q, ST>(p, (int)j, (T)__ldcg(&p.cand_ds[j]), F);
        rewrite_site<Q, ST, ODD>(p, p.cand_site[j], F);
    }
    if (threadIdx.x == 0) p.counters[CNT_DONE] = 0u;
}

// FP64 Delta S of the n records of the last step's list, for
// lbm_last_candidates (the selection may have settled its sites in FP32).
template <int Q, class ST>
__global__ void __launch_bounds__(256) cand_eval_kernel(Params p, unsigned n) {
    const unsigned groups = gridDim.x * (blockDim.x >> 4);
    const unsigned g0 = blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4);
    for (unsigned base = 0; base < n; base += groups) {
        const unsigned j = base + g0;
        const double d = delta_s_group<Q, ST>(p, j, j < n);
        if (j < n && (threadIdx.x & 15) == 0) p.cand_ds[j] = d;
    }
}

// ---------------------------------------------------------------------------
// State transfer, macroscopic fields and entropy.
// ---------------------------------------------------------------------------
template <int Q, class ST>
__global__ void init_kernel(Params p, const double* rho, const double* ux, const double* uy,
                            int eqkind) {
    using T = typename ST::T;
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const int64_t s = (int64_t)y * p.nx + x;
    // in the arithmetic type: FP32 (and 16-bit) storage keeps f* to a few
    // units of its last place either way, and the FP64 form is FP64-pipe
    // bound on GB300 (7x the time of the bytes it moves)
    T feq[Q];
    equilibrium<Q, T>(eqkind, (T)rho[s], (T)ux[s], uy ? (T)uy[s] : T(0), feq);
    typename ST::S* f = (typename ST::S*)p.f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        ST::st(f + (int64_t)i * p.plane + (int64_t)y * p.pitch + x, feq[i], T(L::w(i)));
}

// f = f*(rho, u) with the same rho, u at every site.
template <int Q, class ST>
__global__ void init_uniform_kernel(Params p, double rho, double ux, double uy, int eqkind) {
    using T = typename ST::T;
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    double feq[Q];
    equilibrium<Q, double>(eqkind, rho, ux, uy, feq);
    typename ST::S* f = (typename ST::S*)p.f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        ST::st(f + (int64_t)i * p.plane + (int64_t)y * p.pitch + x, (T)feq[i], T(L::w(i)));
}

template <int Q, class ST, class In>
__global__ void set_state_kernel(Params p, const In* src) {
    using T = typename ST::T;
    using L = Lat<Q>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const int64_t N = (int64_t)p.nx * p.ny, s = (int64_t)y * p.nx + x;
    typename ST::S* f = (typename ST::S*)p.f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        ST::st(f + (int64_t)i * p.plane + (int64_t)y * p.pitch + x, (T)src[i * N + s], T(L::w(i)));
}

template <int Q, class ST>
__device__ __forceinline__ void read_state(const Params& p, int x, int y, bool odd,
                                           typename ST::T* f) {
    using T = typename ST::T;
    if (odd)
        load_general<Q, ST, true>(p, x, y, f);
    else
        load_general<Q, ST, false>(p, x, y, f);
}

template <int Q, class ST, class Out>
__global__ void get_state_kernel(Params p, Out* dst, int odd) {
    using T = typename ST::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    T f[Q];
    read_state<Q, ST>(p, x, y, odd != 0, f);
    const int64_t N = (int64_t)p.nx * p.ny, s = (int64_t)y * p.nx + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[i * N + s] = (Out)f[i];
}

// Diffusive Maxwell walls (Section 8): the wall sites of one step - load
// (streaming), the rule of diffusive_rule, store without collision.  Thread
// k walks the perimeter: bottom row, top row, then the two side columns.
template <class ST, bool ODD>
__global__ void __launch_bounds__(256) diffusive_wall_kernel(Params p) {
    pdl_enter();
    using T = typename ST::T;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int side = p.ny - 2;
    int x, y;
    if (k < p.nx) {
        x = k;
        y = 0;
    } else if (k < 2 * p.nx) {
        x = k - p.nx;
        y = p.ny - 1;
    } else if (k < 2 * p.nx + side) {
        x = 0;
        y = 1 + (k - 2 * p.nx);
    } else if (k < 2 * p.nx + 2 * side) {
        x = p.nx - 1;
        y = 1 + (k - 2 * p.nx - side);
    } else {
        return;
    }
    T f[9];
    load_general<9, ST, ODD>(p, x, y, f);
    diffusive_rule<T>(p, x, y, f);
    store_general<9, ST, ODD>(p, x, y, f);
}

// Control-point probe: one thread appends the velocity of site probe_site
// in the state of parity `odd` (the state a step just produced) to the ring
// buffer; launched after each step only while a probe is set.
template <int Q, class ST>
__global__ void probe_kernel(Params p, int odd) {
    pdl_enter();
    using T = typename ST::T;
    T f[Q], rho, ux, uy;
    const int x = p.probe_site % p.nx, y = p.probe_site / p.nx;
    read_state<Q, ST>(p, x, y, odd != 0, f);
    moments<Q, T>(f, rho, ux, uy);
    const unsigned k = p.counters[CNT_PROBE];
    p.probe_buf[2 * (k % (unsigned)p.probe_cap)] = (double)ux;
    p.probe_buf[2 * (k % (unsigned)p.probe_cap) + 1] = (double)uy;
    p.counters[CNT_PROBE] = k + 1;
}

template <int Q, class ST, class Out>
__global__ void macros_kernel(Params p, Out* rho, Out* u, int odd) {
    using T = typename ST::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    T f[Q];
    read_state<Q, ST>(p, x, y, odd != 0, f);
    double r, a, b;
    if constexpr (sizeof(Out) == 4 && sizeof(T) == 4) {
        // FP32 output from FP32 arithmetic: opposite populations are
        // subtracted first (exactly, while they lie within a factor 2 of
        // each other), so rho u keeps its own relative precision however
        // small u is; the FP64 form is FP64-pipe bound on GB300
        using L = Lat<Q>;
        float rf = f[0], jx = 0.f, jy = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) rf += f[i];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (L::opp(i) <= i) continue;
            const float d = f[i] - f[L::opp(i)];
            if (L::cx(i) > 0) jx += d;
            if (L::cx(i) < 0) jx -= d;
            if (L::cy(i) > 0) jy += d;
            if (L::cy(i) < 0) jy -= d;
        }
        r = rf;
        a = jx / rf;
        b = jy / rf;
    } else {
        double fd[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) fd[i] = (double)f[i];
        moments<Q, double>(fd, r, a, b);
    }
    const int64_t N = (int64_t)p.nx * p.ny, s = (int64_t)y * p.nx + x;
    if (rho) rho[s] = (Out)r;
    if (u) {
        u[s] = (Out)a;
        if (Q == 9) u[N + s] = (Out)b;
    }
}

// H = sum_x sum_i f ln(f / W) (block-reduced, one FP64 atomic per block) and
// the FP64 Delta S field against the equilibrium kind eqkind.
template <int Q, class ST>
__global__ void __launch_bounds__(256) entropy_kernel(Params p, double* H, double* dS, int odd,
                                                     int eqkind) {
    using T = typename ST::T;
    using L = Lat<Q>;
    __shared__ double red[32];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    double h = 0.0;
    if (x < p.nx && y < p.ny) {
        T f[Q];
        read_state<Q, ST>(p, x, y, odd != 0, f);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            double v = (double)f[i];
            if (v > 0.0) h += v * log(v / L::w(i));
        }
        if (dS) dS[(int64_t)y * p.nx + x] = delta_s_fp64<Q, T>(f, eqkind);
    }
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = h;
    __syncthreads();
    if (t < 32) {
        const int nw = (blockDim.x * blockDim.y + 31) >> 5;
        double v = t < nw ? red[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (t == 0) atomicAdd(H, v);
    }
}

// ---------------------------------------------------------------------------
// Host-side launchers (explicitly instantiated per storage format).
// ---------------------------------------------------------------------------
template <class ST>
struct Launch {
    static cudaError_t step(int Q, int coll, bool odd, const Params& p, cudaStream_t s);
    static cudaError_t fixup(int Q, int coll, bool odd, const Params& p, cudaStream_t s, int nsm);
    static cudaError_t prepass(int Q, int coll, bool odd, const Params& p, cudaStream_t s);
    static cudaError_t probe(int Q, bool odd, const Params& p, cudaStream_t s);
    static cudaError_t walls(bool odd, const Params& p, cudaStream_t s);
    static cudaError_t init(int Q, const Params& p, const double* r, const double* ux,
                            const double* uy, int eqkind, cudaStream_t s);
    static cudaError_t init_uniform(int Q, const Params& p, double r, double ux, double uy,
                                    int eqkind, cudaStream_t s);
    static cudaError_t set_state(int Q, const Params& p, const void* src, int dtype, cudaStream_t s);
    static cudaError_t get_state(int Q, const Params& p, void* dst, int dtype, bool odd,
                                 cudaStream_t s);
    static cudaError_t macros(int Q, const Params& p, void* rho, void* u, int dtype, bool odd,
                              cudaStream_t s);
    static cudaError_t entropy(int Q, const Params& p, double* H, double* dS, bool odd, int eqkind,
                               cudaStream_t s);
    static cudaError_t cand_eval(int Q, const Params& p, unsigned n, cudaStream_t s);
};

inline cudaError_t launch_p(void (*k)(Params, int), dim3 g, dim3 b, cudaStream_t s, const Params& p, int a) {
    if (!p.pdl) {
        k<<<g, b, 0, s>>>(p, a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t c = {};
    c.gridDim = g;
    c.blockDim = b;
    c.dynamicSmemBytes = 0;
    c.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = at;
    c.numAttrs = 1;
    return cudaLaunchKernelEx(&c, k, p, a);
}

inline cudaError_t launch_p(void (*k)(Params), dim3 g, dim3 b, cudaStream_t s, const Params& p) {
    if (!p.pdl) {
        k<<<g, b, 0, s>>>(p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t c = {};
    c.gridDim = g;
    c.blockDim = b;
    c.dynamicSmemBytes = 0;
    c.stream = s;
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a[0].val.programmaticStreamSerializationAllowed = 1;
    c.attrs = a;
    c.numAttrs = 1;
    return cudaLaunchKernelEx(&c, k, p);
}

inline dim3 site_grid(const Params& p, dim3 block) {
    return dim3((p.nx + block.x - 1) / block.x, (p.ny + block.y - 1) / block.y);
}

inline dim3 site_block(int Q) { return Q == 3 ? dim3(256, 1) : dim3(kBlockX, kBlockY); }

template <int Q, class ST, int COLL>
cudaError_t launch_step_q(bool odd, const Params& p, cudaStream_t s) {
    // two sites per thread where every row starts on a pair boundary (the
    // padded layouts; a dense layout of odd width takes the per-site kernel).
    if constexpr (Q == 9 && kPairedSites<ST, COLL>) {
        const bool paired = p.pitch % 2 == 0 && p.plane32 % 2 == 0 &&
                            (uintptr_t)p.f % (2 * sizeof(typename ST::S)) == 0;
        if (paired) {
            dim3 b(kVecX, kVecY), g((p.nx + 2 * kVecX - 1) / (2 * kVecX), (p.ny + kVecY - 1) / kVecY);
            return launch_p(odd ? step_kernel_v2<Q, ST, COLL, true> : step_kernel_v2<Q, ST, COLL, false>, g, b,
                            s, p);
        }
    }
    dim3 b = site_block(Q);
    if (Q == 3) {
        // a D1Q3 line has few sites (the 800-site tube): spread them over the
        // SMs in CTAs of as few as 32 threads, so that the ELBM root finder's
        // FP64 chains and the limiter steps run on many SMs at once
        const int nsm = p.pipe_ctas >= 8 ? p.pipe_ctas / 8 : 1;
        int t = ((p.nx + nsm - 1) / nsm + 31) / 32 * 32;
        b = dim3(t < 32 ? 32 : (t > 256 ? 256 : t), 1);
    }
    const dim3 g = site_grid(p, b);
    return launch_p(odd ? step_kernel<Q, ST, COLL, true> : step_kernel<Q, ST, COLL, false>, g, b, s, p);
}

template <int Q, class ST>
cudaError_t launch_step_c(int coll, bool odd, const Params& p, cudaStream_t s) {
    switch (coll) {
        case LBM_LBGK: return launch_step_q<Q, ST, LBM_LBGK>(odd, p, s);
        case LBM_ELBM: return launch_step_q<Q, ST, LBM_ELBM>(odd, p, s);
        case LBM_EHRENFEST: return launch_step_q<Q, ST, LBM_EHRENFEST>(odd, p, s);
        case LBM_POSITIVITY: return launch_step_q<Q, ST, LBM_POSITIVITY>(odd, p, s);
        case LBM_MEDIAN:
            // without a Delta S field the median step is the Ehrenfest one
            // (LBGK and the screen); median_recon_fixup does the rest
            if (p.median_inv != 0.0) return launch_step_q<Q, ST, LBM_EHRENFEST>(odd, p, s);
            return launch_step_q<Q, ST, LBM_MEDIAN>(odd, p, s);
        case LBM_MRT: return launch_step_q<Q, ST, LBM_MRT>(odd, p, s);
        case LBM_SMOOTH: return launch_step_q<Q, ST, LBM_SMOOTH>(odd, p, s);
        case LBM_DOUBLE_MONOTONIC: return launch_step_q<Q, ST, LBM_DOUBLE_MONOTONIC>(odd, p, s);
        case LBM_ENSEMBLE: return launch_step_q<Q, ST, LBM_ENSEMBLE>(odd, p, s);
        case LBM_THRESHOLD: return launch_step_q<Q, ST, LBM_THRESHOLD>(odd, p, s);
        case LBM_MRT2: return launch_step_q<Q, ST, LBM_MRT2>(odd, p, s);
        case LBM_MRT_LIMITER: return launch_step_q<Q, ST, LBM_MRT_LIMITER>(odd, p, s);
        case LBM_ENSEMBLE_LAGGED: return launch_step_q<Q, ST, LBM_ENSEMBLE_LAGGED>(odd, p, s);
    }
    return cudaErrorInvalidValue;
}

template <int Q, class ST>
cudaError_t launch_fixup_q(int coll, bool odd, const Params& p, cudaStream_t s, int nsm) {
    // the candidate count is only known on the device: a fixed grid of one
    // CTA per SM strides over the list
    if (coll == LBM_EHRENFEST)
        return launch_p(odd ? ehrenfest_eval_select<Q, ST, true> : ehrenfest_eval_select<Q, ST, false>, nsm,
                        256, s, p);
    // the field-free median filter takes one candidate per CTA and round:
    // four CTAs per SM, so that thousands of candidates overlap their FP64
    // window evaluations (with few, the CTAs without one exit at once)
    if (coll == LBM_MEDIAN && p.median_inv != 0.0)
        return launch_p(odd ? median_recon_fixup<Q, ST, true> : median_recon_fixup<Q, ST, false>, 4 * nsm, 256,
                        s, p);
    if (coll == LBM_MEDIAN)
        return launch_p(odd ? median_fixup<Q, ST, true> : median_fixup<Q, ST, false>, nsm, 256, s, p);
    if (coll == LBM_THRESHOLD)
        return launch_p(odd ? threshold_eval_select<Q, ST, true> : threshold_eval_select<Q, ST, false>, nsm,
                        256, s, p);
    if (coll == LBM_MRT_LIMITER)
        return launch_p(odd ? mrt_limiter_eval_select<Q, ST, true> : mrt_limiter_eval_select<Q, ST, false>, nsm,
                        256, s, p);
    if (coll == LBM_ENSEMBLE_LAGGED) return launch_p(ensemble_finalize<ST>, 1, 256, s, p);
    return cudaSuccess;
}

template <int Q, class ST>
cudaError_t launch_prepass_q(int coll, bool odd, const Params& p, cudaStream_t s) {
    if (coll != LBM_ENSEMBLE) return cudaSuccess;
    void (*k)(Params) = odd ? ensemble_mean<Q, ST, true> : ensemble_mean<Q, ST, false>;
    // one full wave (the CTAs that fit on the SMs at once) strides over the
    // lattice: a partial second wave would leave SMs idle for its length
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    const int nsm = p.pipe_ctas >= 8 ? p.pipe_ctas / 8 : 1;
    return launch_p(k, dim3(per_sm * nsm), dim3(256), s, p);
}

template <class ST>
cudaError_t Launch<ST>::step(int Q, int coll, bool odd, const Params& p, cudaStream_t s) {
    return Q == 3 ? launch_step_c<3, ST>(coll, odd, p, s) : launch_step_c<9, ST>(coll, odd, p, s);
}

template <class ST>
cudaError_t Launch<ST>::walls(bool odd, const Params& p, cudaStream_t s) {
    const int n = 2 * p.nx + 2 * (p.ny - 2);
    return launch_p(odd ? diffusive_wall_kernel<ST, true> : diffusive_wall_kernel<ST, false>,
                    dim3((n + 255) / 256), dim3(256), s, p);
}

template <class ST>
cudaError_t Launch<ST>::cand_eval(int Q, const Params& p, unsigned n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned g = (n + 15) / 16 < 1024u ? (n + 15) / 16 : 1024u;
    if (Q == 3)
        cand_eval_kernel<3, ST><<<g, 256, 0, s>>>(p, n);
    else
        cand_eval_kernel<9, ST><<<g, 256, 0, s>>>(p, n);
    return cudaGetLastError();
}

template <class ST>
cudaError_t Launch<ST>::probe(int Q, bool odd, const Params& p, cudaStream_t s) {
    return launch_p(Q == 3 ? probe_kernel<3, ST> : probe_kernel<9, ST>, dim3(1), dim3(1), s, p, odd ? 1 : 0);
}

template <class ST>
cudaError_t Launch<ST>::prepass(int Q, int coll, bool odd, const Params& p, cudaStream_t s) {
    return Q == 3 ? launch_prepass_q<3, ST>(coll, odd, p, s) : launch_prepass_q<9, ST>(coll, odd, p, s);
}

template <class ST>
cudaError_t Launch<ST>::fixup(int Q, int coll, bool odd, const Params& p, cudaStream_t s, int nsm) {
    return Q == 3 ? launch_fixup_q<3, ST>(coll, odd, p, s, nsm)
                  : launch_fixup_q<9, ST>(coll, odd, p, s, nsm);
}

template <class ST>
cudaError_t Launch<ST>::init(int Q, const Params& p, const double* r, const double* ux,
                             const double* uy, int eqkind, cudaStream_t s) {
    dim3 b = site_block(Q), g = site_grid(p, b);
    if (Q == 3)
        init_kernel<3, ST><<<g, b, 0, s>>>(p, r, ux, uy, eqkind);
    else
        init_kernel<9, ST><<<g, b, 0, s>>>(p, r, ux, uy, eqkind);
    return cudaGetLastError();
}

template <class ST>
cudaError_t Launch<ST>::init_uniform(int Q, const Params& p, double r, double ux, double uy,
                                     int eqkind, cudaStream_t s) {
    dim3 b = site_block(Q), g = site_grid(p, b);
    if (Q == 3)
        init_uniform_kernel<3, ST><<<g, b, 0, s>>>(p, r, ux, uy, eqkind);
    else
        init_uniform_kernel<9, ST><<<g, b, 0, s>>>(p, r, ux, uy, eqkind);
    return cudaGetLastError();
}

template <class ST>
cudaError_t Launch<ST>::set_state(int Q, const Params& p, const void* src, int dtype,
                                  cudaStream_t s) {
    dim3 b = site_block(Q), g = site_grid(p, b);
    if (dtype == LBM_DTYPE_F64) {
        if (Q == 3)
            set_state_kernel<3, ST, double><<<g, b, 0, s>>>(p, (const double*)src);
        else
            set_state_kernel<9, ST, double><<<g, b, 0, s>>>(p, (const double*)src);
    } else {
        if (Q == 3)
            set_state_kernel<3, ST, float><<<g, b, 0, s>>>(p, (const float*)src);
        else
            set_state_kernel<9, ST, float><<<g, b, 0, s>>>(p, (const float*)src);
    }
    return cudaGetLastError();
}

template <class ST>
cudaError_t Launch<ST>::get_state(int Q, const Params& p, void* dst, int dtype, bool odd,
                                  cudaStream_t s) {
    dim3 b = site_block(Q), g = site_grid(p, b);
    if (dtype == LBM_DTYPE_F64) {
        if (Q == 3)
            get_state_kernel<3, ST, double><<<g, b, 0, s>>>(p, (double*)dst, odd);
        else
            get_state_kernel<9, ST, double><<<g, b, 0, s>>>(p, (double*)dst, odd);
    } else {
        if (Q == 3)
            get_state_kernel<3, ST, float><<<g, b, 0, s>>>(p, (float*)dst, odd);
        else
            get_state_kernel<9, ST, float><<<g, b, 0, s>>>(p, (float*)dst, odd);
    }
    return cudaGetLastError();
}

template <class ST>
cudaError_t Launch<ST>::macros(int Q, const Params& p, void* rho, void* u, int dtype, bool odd,
                               cudaStream_t s) {
    dim3 b = site_block(Q), g = site_grid(p, b);
    if (dtype == LBM_DTYPE_F64) {
        if (Q == 3)
            macros_kernel<3, ST, double><<<g, b, 0, s>>>(p, (double*)rho, (double*)u, odd);
        else
            macros_kernel<9, ST, double><<<g, b, 0, s>>>(p, (double*)rho, (double*)u, odd);
    } else {
        if (Q == 3)
            macros_kernel<3, ST, float><<<g, b, 0, s>>>(p, (float*)rho, (float*)u, odd);
        else
            macros_kernel<9, ST, float><<<g, b, 0, s>>>(p, (float*)rho, (float*)u, odd);
    }
    return cudaGetLastError();
}

template <class ST>
cudaError_t Launch<ST>::entropy(int Q, const Params& p, double* H, double* dS, bool odd,
                                int eqkind, cudaStream_t s) {
    dim3 b = site_block(Q), g = site_grid(p, b);
    if (Q == 3)
        entropy_kernel<3, ST><<<g, b, 0, s>>>(p, H, dS, odd, eqkind);
    else
        entropy_kernel<9, ST><<<g, b, 0, s>>>(p, H, dS, odd, eqkind);
    return cudaGetLastError();
}

}  // namespace lbm
