// Reverse-mode (adjoint) kernels of the step for the LBGK, Ehrenfest,
// median-filter and positivity collisions, on dense natural-layout states
// f[i][y][x].
//
// One step is f_{t+1} = P(C(f_t)): C the collision at every site, P the
// streaming with half-way bounce-back and the moving-lid term
// -6 W_i v_ix U on links through the top wall.  Every branch of these
// collisions has the form F = f* + psi (f - f*):
//   LBGK (Eq. CollisionIntegral)         psi = 1 - 2 beta
//   Ehrenfest step (Section 4)           psi = 0
//   median filter (Section 4.4, entrHom) psi = (1 - 2 beta) sqrt(M / C), C the
//                                        site's Delta S, M that of the window
//                                        site m holding the lower median
//   positivity rule (Section 4, StrLine) psi = f*_k / (f*_k - f_k), k the
//                                        population that binds the rule
// and the selection of each step (which branch, m, k) is held fixed.  Given
// lambda_{t+1} = dJ/df_{t+1}:
//   Lambda = P^T lambda_{t+1}:  Lambda_i(x) = lambda_{t+1, i}(x + v_i), or
//     lambda_{t+1, opp(i)}(x) for a wall link (which also adds
//     lambda_{t+1, opp(i)}(x) (-6 W_i v_ix) to dJ/dU on the lid);
//   lambda_t,j = (1 - psi) a_j + psi Lambda_j + g dpsi/df_j,
//     a_j = sum_i Lambda_i df*_i/df_j,  g = sum_i Lambda_i (f_i - f*_i);
//   dJ/dbeta += g dpsi/dbeta (-2 for LBGK, -2 sqrt(M / C) for the median,
//     0 for the Ehrenfest step and the positivity rule);
//   the median's psi also depends on f at m: lambda_t(m) += g dpsi/df(m).
// df*/df_j = df*/drho + df*/du_x (v_jx - u_x)/rho + df*/du_y (v_jy - u_y)/rho.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

struct AdjGeo {
    int nx, ny, periodic_x, periodic_y;
    int eq;  // equilibrium kind
    double beta;
};

// 1D equilibrium (per unit density) and its derivative in u, both forms
// a -+ u/2, 1 - 2a: a' = u (polynomial) or u / sqrt(1 + 3u^2) (entropic).
template <class T>
__device__ __forceinline__ void eq1d_d(int kind, T u, T* phi, T* dphi) {
    if (kind == LBM_EQ_ENTROPIC) {
        eq1d_entropic<T>(u, phi[0], phi[1], phi[2]);
        const T da = u / sqrt(T(1) + T(3) * u * u);
        dphi[0] = da - T(0.5);
        dphi[1] = T(-2) * da;
        dphi[2] = da + T(0.5);
    } else {
        eq1d_poly<T>(u, phi[0], phi[1], phi[2]);
        dphi[0] = u - T(0.5);
        dphi[1] = T(-2) * u;
        dphi[2] = u + T(0.5);
    }
}

// f*, df*/drho, df*/dux, df*/duy at one site.
template <int Q, class T>
__device__ __forceinline__ void eq_partials(int kind, T rho, T ux, T uy, T* feq, T* dr, T* dx, T* dy) {
    using L = Lat<Q>;
    if (Q == 9 && kind == LBM_EQ_POLY_STD) {
        const T uu = ux * ux + uy * uy;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T cxi = T(L::cx(i)), cyi = T(L::cy(i)), cu = cxi * ux + cyi * uy, w = T(L::w(i));
            dr[i] = w * (T(1) + T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
            feq[i] = rho * dr[i];
            dx[i] = w * rho * (T(3) * cxi + T(9) * cu * cxi - T(3) * ux);
            dy[i] = w * rho * (T(3) * cyi + T(9) * cu * cyi - T(3) * uy);
        }
        return;
    }
    T px[3], dpx[3], py[3] = {T(0), T(1), T(0)}, dpy[3] = {T(0), T(0), T(0)};
    eq1d_d<T>(kind, ux, px, dpx);
    if (Q == 9) eq1d_d<T>(kind, uy, py, dpy);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int a = L::cx(i) + 1, b = L::cy(i) + 1;
        dr[i] = px[a] * py[b];
        feq[i] = rho * dr[i];
        dx[i] = rho * dpx[a] * py[b];
        dy[i] = rho * px[a] * dpy[b];
    }
}

template <int Q, class T>
__device__ __forceinline__ void dense_site(const T* a, int64_t N, int64_t s, T* out) {
#pragma unroll
    for (int i = 0; i < Q; ++i) out[i] = a[(int64_t)i * N + s];
}

// Block-wide sum of up to two doubles into acc[k] (one atomic per block).
__device__ __forceinline__ void block_add2(double v0, double v1, double* acc0, double* acc1) {
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    const int t = threadIdx.x, w = t >> 5;
    if ((t & 31) == 0) {
        red[0][w] = v0;
        red[1][w] = v1;
    }
    __syncthreads();
    if (t < 32) {
        const int nw = (blockDim.x + 31) >> 5;
        double a = t < nw ? red[0][t] : 0.0, b = t < nw ? red[1][t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (t == 0) {
            if (acc0 && a != 0.0) atomicAdd(acc0, a);
            if (acc1 && b != 0.0) atomicAdd(acc1, b);
        }
    }
}

// Seed of J = 1/2 sum rho |u|^2: lambda_j = v_j . u - |u|^2 / 2, and J.
template <int Q, class T>
__global__ void __launch_bounds__(256) adj_seed_ke(AdjGeo g, const T* __restrict__ f, T* lam,
                                                  double* J) {
    using L = Lat<Q>;
    const int64_t N = (int64_t)g.nx * g.ny;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (s < N) {
        T fs[Q], rho, ux, uy;
        dense_site<Q, T>(f, N, s, fs);
        moments<Q, T>(fs, rho, ux, uy);
        const T uu = ux * ux + uy * uy;
#pragma unroll
        for (int j = 0; j < Q; ++j) lam[(int64_t)j * N + s] = T(L::cx(j)) * ux + T(L::cy(j)) * uy - T(0.5) * uu;
        e = 0.5 * (double)rho * (double)uu;
    }
    block_add2(e, 0.0, J, nullptr);
}

// The adjoint kernels hold the rare FP64 branch work (median Delta S
// gradients) in out-of-line functions and are compiled for four resident
// CTAs per SM (two in FP64): the rare work spills instead of setting every site's
// register allocation (without the cap a kernel takes over 200 registers).
template <class T>
constexpr int kAdjMinBlocks = sizeof(T) == 8 ? 2 : 4;

// Branch of a site in one step (the int recorded per site and step).
enum { AUX_LBGK = -1, AUX_FSTAR = -2, AUX_POS0 = -3 };  // AUX_POS0 - k; m >= 0: median

// Delta S of one site in FP64 (the cancellation-free form of Eq. DelS) and
// its gradient dDelta S/df_j = ln(f_j/f*_j) + 1 - sum_i (f_i/f*_i) df*_i/df_j.
// +inf (gradient 0) with a non-positive population.
template <int Q>
__device__ __noinline__ double delta_s_grad(int eqkind, const double* f, double* grad) {
    using L = Lat<Q>;
    double rho, ux, uy, feq[Q], dr[Q], dx[Q], dy[Q];
    moments<Q, double>(f, rho, ux, uy);
    eq_partials<Q, double>(eqkind, rho, ux, uy, feq, dr, dx, dy);
    double ds = 0.0;
    bool neg = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        neg |= !(f[i] > 0.0) || !(feq[i] > 0.0);
        ds += feq[i] * gfun_d((f[i] - feq[i]) / feq[i]);
    }
    // sum_i (f_i / f*_i) df*_i/df_j = S0 + (v_jx - u_x) Sx / rho + (v_jy - u_y) Sy / rho
    double r[Q], S0 = 0.0, Sx = 0.0, Sy = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        r[i] = f[i] / feq[i];
        S0 += r[i] * dr[i];
        Sx += r[i] * dx[i];
        Sy += r[i] * dy[i];
    }
    const double ir = 1.0 / rho;
#pragma unroll
    for (int j = 0; j < Q; ++j)
        grad[j] = neg ? 0.0 : log(r[j]) + 1.0 - (S0 + (L::cx(j) - ux) * ir * Sx + (L::cy(j) - uy) * ir * Sy);
    return neg ? __longlong_as_double(0x7ff0000000000000ULL) : ds;
}

template <int Q, class T>
__device__ __forceinline__ void dense_site_d(const T* a, int64_t N, int64_t s, double* out) {
#pragma unroll
    for (int i = 0; i < Q; ++i) out[i] = (double)a[(int64_t)i * N + s];
}

// Records the branch of every site of one recomputed step (aux cleared to
// AUX_LBGK beforehand), from the step's candidate list (Ehrenfest, median:
// the selection the step made) or, for the positivity rule, by the step's own
// test on the dense pre-collision state f (the same device functions in the
// same precision, so the same decision).  The median's window site m: the
// lower median of the clipped window's FP64 Delta S, ties by site index.
template <int Q, class T>
__global__ void __launch_bounds__(256, kAdjMinBlocks<T>) adj_record(Params p, int coll, int cslot, const T* __restrict__ f,
                                                 int* __restrict__ aux) {
    const int64_t N = (int64_t)p.nx * p.ny;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    if (coll == LBM_POSITIVITY) {
        for (int64_t s = tid; s < N; s += nt) {
            T fs[Q], feq[Q], F[Q], rho, ux, uy;
#pragma unroll
            for (int i = 0; i < Q; ++i) fs[i] = f[(int64_t)i * N + s];
            moments<Q, T>(fs, rho, ux, uy);
            equilibrium<Q, T>(p.eq, rho, ux, uy, feq);
            lbgk<Q, T>(fs, feq, sizeof(T) == 8 ? T(p.beta) : T(p.beta_f), F);
            T lam = T(1);
            int k = -1;
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (F[i] < T(0)) {
                    const T l = feq[i] / (feq[i] - F[i]);
                    if (l < lam) {  // the first of equal values, as positivity()
                        lam = l;
                        k = i;
                    }
                }
            if (k >= 0) aux[s] = AUX_POS0 - k;
        }
        return;
    }
    unsigned M = p.counters[cslot];
    if (M > (unsigned)p.cand_cap) M = (unsigned)p.cand_cap;
    if (coll == LBM_EHRENFEST) {
        for (int64_t j = tid; j < (int64_t)M; j += nt)
            if (p.cand_sel[j] && p.cand_ds[j] > p.delta) aux[p.cand_site[j]] = AUX_FSTAR;
        return;
    }
    // median: one warp per selected candidate, one lane per window site
    // (lane l: offset (l % 3 - 1, l / 3 - ry), the window's scan order);
    // the first lane sorts the values and keeps the window site of the
    // lower median
    const int lane = threadIdx.x & 31;
    const int ry = Q == 9 ? 1 : 0;
    for (int64_t j = tid >> 5; j < (int64_t)M; j += nt >> 5) {
        if (!p.cand_sel[j]) continue;  // the same j on every lane
        const int site = p.cand_site[j];
        const int x = site % p.nx, y = site / p.nx;
        int q = -1;
        double d = 0.0;
        if (lane < 3 * (2 * ry + 1)) {
            int xx = x + lane % 3 - 1, yy = y + lane / 3 - ry;
            if (p.periodic_x) xx = xx < 0 ? xx + p.nx : (xx >= p.nx ? xx - p.nx : xx);
            if (p.periodic_y) yy = yy < 0 ? yy + p.ny : (yy >= p.ny ? yy - p.ny : yy);
            if (xx >= 0 && xx < p.nx && yy >= 0 && yy < p.ny) {
                q = yy * p.nx + xx;
                double fq[Q], g[Q];
                dense_site_d<Q, T>(f, N, q, fq);
                d = delta_s_grad<Q>(p.eq, fq, g);
            }
        }
        int w[9];
        double v[9];
        int n = 0;
#pragma unroll
        for (int l = 0; l < 3 * (2 * ry + 1); ++l) {
            const int ql = __shfl_sync(0xffffffffu, q, l);
            const double dl = __shfl_sync(0xffffffffu, d, l);
            if (ql < 0) continue;
            int k = n++;
            while (k > 0 && (v[k - 1] > dl || (v[k - 1] == dl && w[k - 1] > ql))) {  // ascending
                v[k] = v[k - 1];
                w[k] = w[k - 1];
                --k;
            }
            v[k] = dl;
            w[k] = ql;
        }
        if (lane == 0) aux[site] = w[(n - 1) / 2];
    }
}

// The positivity and median branches of the adjoint step at site s (psi,
// dpsi/dbeta, dpsi/df_j and the median's cross-term coefficient w), out of
// line: they are rare, and the median's FP64 Delta S gradients would
// otherwise set the register allocation of every site's adjoint step.
template <int Q, class T>
struct AdjBranch {
    T psi, dpsi_db, dpsi[Q];
    double w;
};

template <int Q, class T>
__device__ __noinline__ AdjBranch<Q, T> adj_branch(AdjGeo g, const T* __restrict__ f, int64_t N, int64_t s,
                                                   int br, T gs) {
    using L = Lat<Q>;
    AdjBranch<Q, T> b;
    T fs[Q], feq[Q], dr[Q], dx[Q], dy[Q], rho, ux, uy;
    dense_site<Q, T>(f, N, s, fs);
    moments<Q, T>(fs, rho, ux, uy);
    eq_partials<Q, T>(g.eq, rho, ux, uy, feq, dr, dx, dy);
    const T inv = T(1) / rho;
    const T c = T(1) - T(2) * T(g.beta);
    b.w = 0.0;
#pragma unroll
    for (int j = 0; j < Q; ++j) b.dpsi[j] = T(0);
    if (br <= AUX_POS0) {
        // psi = f*_k / (f*_k - f_k), independent of beta
        const int k = AUX_POS0 - br;
        T fk = T(0), ek = T(0), drk = T(0), dxk = T(0), dyk = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (i == k) {
                fk = fs[i];
                ek = feq[i];
                drk = dr[i];
                dxk = dx[i];
                dyk = dy[i];
            }
        const T D = ek - fk;
        b.psi = ek / D;
        b.dpsi_db = T(0);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const T dfk = drk + dxk * (T(L::cx(j)) - ux) * inv + dyk * (T(L::cy(j)) - uy) * inv;
            b.dpsi[j] = (-fk * dfk + (j == k ? ek : T(0))) / (D * D);
        }
        return b;
    }
    // psi = c sqrt(M / C): C and its gradient here, M at window site br (FP64)
    double fd[Q], gC[Q], fm[Q], gM[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fd[i] = (double)fs[i];
    const double C = delta_s_grad<Q>(g.eq, fd, gC);
    dense_site_d<Q, T>(f, N, br, fm);
    const double Mv = delta_s_grad<Q>(g.eq, fm, gM);
    const double phi = isinf(C) ? 0.0 : sqrt(Mv / C);
    b.psi = T(c * T(phi));
    b.dpsi_db = T(-2.0 * phi);
    if (!isinf(C) && Mv > 0.0) {
#pragma unroll
        for (int j = 0; j < Q; ++j) b.dpsi[j] = T(-(double)c * phi / (2.0 * C) * gC[j]);
        b.w = (double)gs * (double)c * phi / (2.0 * Mv);
    }
    return b;
}

// lambda_t from lambda_{t+1} (see the header), with dJ/dU in acc[0] and
// dJ/dbeta in acc[1]; aux (NULL: every site LBGK) holds each site's branch.
// For a median site the coefficient w = g (1 - 2 beta) sqrt(M / C) / (2 M) of
// its cross term goes to wbuf[s] (adj_median_cross adds it at m).
template <int Q, class T>
__global__ void __launch_bounds__(256, kAdjMinBlocks<T>)
    adj_step(AdjGeo g, const T* __restrict__ f, const int* __restrict__ aux, const T* __restrict__ lam_in,
             T* __restrict__ lam_out, double* acc, double* __restrict__ wbuf) {
    using L = Lat<Q>;
    const int64_t N = (int64_t)g.nx * g.ny;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dU = 0.0, dB = 0.0;
    if (s < N) {
        const int x = (int)s % g.nx, y = (int)s / g.nx;  // N < 2^31
        T Lam[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int tx = x + L::cx(i), ty = y + L::cy(i);
            if (g.periodic_x) tx = tx < 0 ? tx + g.nx : (tx >= g.nx ? tx - g.nx : tx);
            if (g.periodic_y) ty = ty < 0 ? ty + g.ny : (ty >= g.ny ? ty - g.ny : ty);
            if (tx >= 0 && tx < g.nx && ty >= 0 && ty < g.ny) {
                Lam[i] = lam_in[(int64_t)i * N + (int64_t)ty * g.nx + tx];
            } else {
                Lam[i] = lam_in[(int64_t)L::opp(i) * N + s];
                if (ty >= g.ny) dU += (double)Lam[i] * (-6.0 * L::w(i) * L::cx(i));
            }
        }
        T fs[Q], feq[Q], dr[Q], dx[Q], dy[Q], rho, ux, uy;
        dense_site<Q, T>(f, N, s, fs);
        moments<Q, T>(fs, rho, ux, uy);
        eq_partials<Q, T>(g.eq, rho, ux, uy, feq, dr, dx, dy);
        T A = T(0), Bx = T(0), By = T(0), gs = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            A += Lam[i] * dr[i];
            Bx += Lam[i] * dx[i];
            By += Lam[i] * dy[i];
            gs += Lam[i] * (fs[i] - feq[i]);
        }
        const T inv = T(1) / rho;
        const int br = aux ? aux[s] : AUX_LBGK;
        T psi = T(1) - T(2) * T(g.beta), dpsi_db = T(-2), dpsi[Q];
#pragma unroll
        for (int j = 0; j < Q; ++j) dpsi[j] = T(0);
        if (br == AUX_FSTAR) {
            psi = T(0);
            dpsi_db = T(0);
        } else if (br != AUX_LBGK) {
            const AdjBranch<Q, T> b = adj_branch<Q, T>(g, f, N, s, br, gs);
            psi = b.psi;
            dpsi_db = b.dpsi_db;
#pragma unroll
            for (int j = 0; j < Q; ++j) dpsi[j] = b.dpsi[j];
            if (br >= 0) wbuf[s] = b.w;
        }
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const T a = A + Bx * (T(L::cx(j)) - ux) * inv + By * (T(L::cy(j)) - uy) * inv;
            lam_out[(int64_t)j * N + s] = (T(1) - psi) * a + psi * Lam[j] + gs * dpsi[j];
        }
        dB = (double)gs * (double)dpsi_db;
    }
    block_add2(dU, dB, acc, acc + 1);
}

// The median's cross term: a selected site s with window site m = aux[s]
// adds wbuf[s] dM/df(m) to lambda_t(m) (after adj_step has written it).
template <int Q, class T>
__device__ __noinline__ void adj_cross_site(AdjGeo g, const T* __restrict__ f, int64_t N, int m, double w,
                                            T* lam_out) {
    double fm[Q], gM[Q];
    dense_site_d<Q, T>(f, N, m, fm);
    delta_s_grad<Q>(g.eq, fm, gM);
#pragma unroll
    for (int j = 0; j < Q; ++j) atomicAdd(&lam_out[(int64_t)j * N + m], T(w * gM[j]));
}

template <int Q, class T>
__global__ void __launch_bounds__(256, kAdjMinBlocks<T>) adj_median_cross(AdjGeo g, const T* __restrict__ f,
                                                       const int* __restrict__ aux,
                                                       const double* __restrict__ wbuf, T* lam_out) {
    const int N = g.nx * g.ny;  // < 2^31
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int m = aux[s];
        if (m < 0) continue;
        const double w = wbuf[s];
        if (w != 0.0) adj_cross_site<Q, T>(g, f, N, m, w, lam_out);
    }
}

template <class T, class U>
__global__ void convert_kernel(const T* __restrict__ a, U* __restrict__ b, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        b[k] = (U)a[k];
}

template <class T>
struct AdjLaunch {
    static cudaError_t seed(int Q, const AdjGeo& g, const T* f, T* lam, double* J, cudaStream_t s) {
        const int64_t N = (int64_t)g.nx * g.ny;
        const unsigned blocks = (unsigned)((N + 255) / 256);
        if (Q == 3)
            adj_seed_ke<3, T><<<blocks, 256, 0, s>>>(g, f, lam, J);
        else
            adj_seed_ke<9, T><<<blocks, 256, 0, s>>>(g, f, lam, J);
        return cudaGetLastError();
    }
    static cudaError_t step(int Q, const AdjGeo& g, const T* f, const int* aux, const T* lin, T* lout,
                            double* acc, double* wbuf, bool median, cudaStream_t s) {
        const int64_t N = (int64_t)g.nx * g.ny;
        const unsigned blocks = (unsigned)((N + 255) / 256);
        if (Q == 3)
            adj_step<3, T><<<blocks, 256, 0, s>>>(g, f, aux, lin, lout, acc, wbuf);
        else
            adj_step<9, T><<<blocks, 256, 0, s>>>(g, f, aux, lin, lout, acc, wbuf);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || !median) return e;
        if (Q == 3)
            adj_median_cross<3, T><<<blocks, 256, 0, s>>>(g, f, aux, wbuf, lout);
        else
            adj_median_cross<9, T><<<blocks, 256, 0, s>>>(g, f, aux, wbuf, lout);
        return cudaGetLastError();
    }
    static cudaError_t record(int Q, const Params& p, int coll, int cslot, const T* f, int* aux, int nsm,
                              cudaStream_t s) {
        const int64_t N = (int64_t)p.nx * p.ny;
        const unsigned blocks =
            coll == LBM_POSITIVITY ? (unsigned)std::min<int64_t>((N + 255) / 256, 8 * nsm) : (unsigned)nsm;
        if (Q == 3)
            adj_record<3, T><<<blocks, 256, 0, s>>>(p, coll, cslot, f, aux);
        else
            adj_record<9, T><<<blocks, 256, 0, s>>>(p, coll, cslot, f, aux);
        return cudaGetLastError();
    }
    template <class U>
    static cudaError_t convert(const T* a, U* b, int64_t n, cudaStream_t s) {
        const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
        convert_kernel<T, U><<<blocks, 256, 0, s>>>(a, b, n);
        return cudaGetLastError();
    }
};

}  // namespace lbm
