// Reverse-mode (adjoint) kernels of the step for the LBGK and Ehrenfest
// collisions, on dense natural-layout states f[i][y][x].
//
// One step is f_{t+1} = P(C(f_t)): C the collision at every site, P the
// streaming with half-way bounce-back and the moving-lid term
// -6 W_i v_ix U on links through the top wall.  Given lambda_{t+1} =
// dJ/df_{t+1}:
//   Lambda = P^T lambda_{t+1}:  Lambda_i(x) = lambda_{t+1, i}(x + v_i), or
//     lambda_{t+1, opp(i)}(x) for a wall link (which also adds
//     lambda_{t+1, opp(i)}(x) (-6 W_i v_ix) to dJ/dU on the lid);
//   lambda_t = (dC/df)^T Lambda, with dC/df = (1 - 2 beta) I + 2 beta df*/df for
//     LBGK sites and df*/df for the sites the Ehrenfest step sent to f*
//     (the selection of that step is held fixed);
//   dJ/dbeta += Lambda . 2 (f* - f) at LBGK sites.
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

// Sites the Ehrenfest step of this parity sent to f* (from its candidate list).
template <int Q>
__global__ void adj_mask(Params p, int cslot, unsigned char* mask) {
    unsigned M = p.counters[cslot];
    if (M > (unsigned)p.cand_cap) M = (unsigned)p.cand_cap;
    for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
        if (p.cand_sel[j] && p.cand_ds[j] > p.delta) mask[p.cand_site[j]] = 1;
}

// lambda_t from lambda_{t+1} (see the header), with dJ/dU in acc[0] and
// dJ/dbeta in acc[1].
template <int Q, class T>
__global__ void __launch_bounds__(256)
    adj_step(AdjGeo g, const T* __restrict__ f, const unsigned char* __restrict__ mask,
             const T* __restrict__ lam_in, T* __restrict__ lam_out, double* acc) {
    using L = Lat<Q>;
    const int64_t N = (int64_t)g.nx * g.ny;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dU = 0.0, dB = 0.0;
    if (s < N) {
        const int x = (int)(s % g.nx), y = (int)(s / g.nx);
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
        T A = T(0), Bx = T(0), By = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            A += Lam[i] * dr[i];
            Bx += Lam[i] * dx[i];
            By += Lam[i] * dy[i];
        }
        const T inv = T(1) / rho;
        const bool sel = mask && mask[s];
        const T om = T(2) * T(g.beta);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const T a = A + Bx * (T(L::cx(j)) - ux) * inv + By * (T(L::cy(j)) - uy) * inv;
            lam_out[(int64_t)j * N + s] = sel ? a : (T(1) - om) * Lam[j] + om * a;
        }
        if (!sel) {
            T b = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) b += Lam[i] * (feq[i] - fs[i]);
            dB = 2.0 * (double)b;
        }
    }
    block_add2(dU, dB, acc, acc + 1);
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
    static cudaError_t step(int Q, const AdjGeo& g, const T* f, const unsigned char* mask,
                            const T* lin, T* lout, double* acc, cudaStream_t s) {
        const int64_t N = (int64_t)g.nx * g.ny;
        const unsigned blocks = (unsigned)((N + 255) / 256);
        if (Q == 3)
            adj_step<3, T><<<blocks, 256, 0, s>>>(g, f, mask, lin, lout, acc);
        else
            adj_step<9, T><<<blocks, 256, 0, s>>>(g, f, mask, lin, lout, acc);
        return cudaGetLastError();
    }
    static cudaError_t mask(int Q, const Params& p, int cslot, unsigned char* m, int nsm, cudaStream_t s) {
        if (Q == 3)
            adj_mask<3><<<nsm, 256, 0, s>>>(p, cslot, m);
        else
            adj_mask<9><<<nsm, 256, 0, s>>>(p, cslot, m);
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
