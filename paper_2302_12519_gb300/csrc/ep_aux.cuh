// ep_aux.cuh -- set-up, diagnostic and reduction kernels of the voxel electrophysiology step.
#pragma once

#include "ep_common.cuh"

namespace gbep {

// ---------------------------------------------------------------------------
// Setup and diagnostic kernels: one thread per voxel, vertices recomputed
// from global memory (8x redundant, used once at setup or for checking).
// ---------------------------------------------------------------------------

// Static data of vertex (I, J, K): valid-pair counts, nT and M = sum f f^T.
__device__ inline void vertex_static(int nx, int ny, int nz, const ushort4 *rec, int I, int J, int K,
                                     int cnt[3], int &nT, double M[6], bool T[2][2][2])
{
    double f[2][2][2][3];
    for (int u = 0; u < 2; ++u)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s) {
                const int i = I - 1 + s, j = J - 1 + t, k = K - 1 + u;
                bool in = i >= 0 && j >= 0 && k >= 0 && i < nx && j < ny && k < nz;
                T[u][t][s] = false;
                f[u][t][s][0] = f[u][t][s][1] = f[u][t][s][2] = 0.0;
                if (in) {
                    const ushort4 r = rec[(long long)i + (long long)nx * ((long long)j + (long long)ny * k)];
                    if (rec_tissue(r)) {
                        T[u][t][s] = true;
                        f[u][t][s][0] = h2f(r.x); f[u][t][s][1] = h2f(r.y); f[u][t][s][2] = h2f(r.z);
                    }
                }
            }
    nT = 0;
    for (int i = 0; i < 6; ++i) M[i] = 0.0;
    cnt[0] = cnt[1] = cnt[2] = 0;
    for (int u = 0; u < 2; ++u)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s) {
                if (!T[u][t][s]) continue;
                const double *g = f[u][t][s];
                ++nT;
                M[0] += g[0] * g[0]; M[1] += g[1] * g[1]; M[2] += g[2] * g[2];
                M[3] += g[0] * g[1]; M[4] += g[0] * g[2]; M[5] += g[1] * g[2];
            }
    for (int o1 = 0; o1 < 2; ++o1)
        for (int o2 = 0; o2 < 2; ++o2) {
            cnt[0] += T[o2][o1][0] && T[o2][o1][1];
            cnt[1] += T[o2][0][o1] && T[o2][1][o1];
            cnt[2] += T[0][o2][o1] && T[1][o2][o1];
        }
}

// Dhat_q = sum over the 8 vertices of q of c^T Shat c, c_a = +-T(partner) r_a,
// Shat = nT sT I + dS M; D_q = Dhat_q / (8 dx^2).  Writes the fp16 record.
__global__ void k_build_records(int nx, int ny, int nz, const float *fib, const uint8_t *mask,
                                ushort4 *rec)
{
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        ushort4 r;
        if (mask[q]) {
            r.x = __half_as_ushort(__float2half_rn(fib[3 * q + 0]));
            r.y = __half_as_ushort(__float2half_rn(fib[3 * q + 1]));
            r.z = __half_as_ushort(__float2half_rn(fib[3 * q + 2]));
            r.w = 0;   // 1/Dhat filled by k_build_diag
        } else {
            r.x = r.y = r.z = 0;
            r.w = kNonTissue;
        }
        rec[q] = r;
    }
}

__global__ void k_build_diag(int nx, int ny, int nz, double sT, double dS, const ushort4 *rec,
                             ushort4 *rec_out)
{
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        ushort4 r = rec[q];
        if (!rec_tissue(r)) { rec_out[q] = r; continue; }
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
        double D = 0.0;
        for (int u = 0; u < 2; ++u)
            for (int t = 0; t < 2; ++t)
                for (int s = 0; s < 2; ++s) {
                    int cnt[3], nT;
                    double M[6];
                    bool T[2][2][2];
                    vertex_static(nx, ny, nz, rec, i + s, j + t, k + u, cnt, nT, M, T);
                    // q sits at block offset (1-s, 1-t, 1-u); partner along a flips that offset
                    const int os = 1 - s, ot = 1 - t, ou = 1 - u;
                    double c[3];
                    c[0] = T[ou][ot][1 - os] && cnt[0] ? (os ? 1.0 : -1.0) / cnt[0] : 0.0;
                    c[1] = T[ou][1 - ot][os] && cnt[1] ? (ot ? 1.0 : -1.0) / cnt[1] : 0.0;
                    c[2] = T[1 - ou][ot][os] && cnt[2] ? (ou ? 1.0 : -1.0) / cnt[2] : 0.0;
                    const double iso = sT * nT;
                    const double S[3][3] = {{iso + dS * M[0], dS * M[3], dS * M[4]},
                                            {dS * M[3], iso + dS * M[1], dS * M[5]},
                                            {dS * M[4], dS * M[5], iso + dS * M[2]}};
                    for (int x = 0; x < 3; ++x)
                        for (int y = 0; y < 3; ++y) D += c[x] * S[x][y] * c[y];
                }
        r.w = D > 0.0 ? __half_as_ushort(__float2half_rn((float)(1.0 / D))) : (unsigned short)0;
        rec_out[q] = r;
    }
}

// Diagnostic: L u by visiting the 8 vertices of each voxel (independent of
// the z-march kernel's data movement).
template <typename real>
__global__ void k_apply_simple(int nx, int ny, int nz, const ushort4 *rec, const real *u, double sT, double dS,
                               double C, real *out)
{
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        if (!rec_tissue(rec[q])) { out[q] = 0; continue; }
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
        double acc = 0.0;
        for (int uu = 0; uu < 2; ++uu)
            for (int t = 0; t < 2; ++t)
                for (int s = 0; s < 2; ++s) {
                    const int I = i + s, J = j + t, K = k + uu;
                    int cnt[3], nT;
                    double M[6];
                    bool T[2][2][2];
                    vertex_static(nx, ny, nz, rec, I, J, K, cnt, nT, M, T);
                    double val[2][2][2];
                    for (int a2 = 0; a2 < 2; ++a2)
                        for (int b2 = 0; b2 < 2; ++b2)
                            for (int c2 = 0; c2 < 2; ++c2) {
                                const int ii = I - 1 + c2, jj = J - 1 + b2, kk = K - 1 + a2;
                                val[a2][b2][c2] = T[a2][b2][c2] ? (double)u[(long long)ii + (long long)nx * ((long long)jj + (long long)ny * kk)] : 0.0;
                            }
                    double g[3] = {0, 0, 0};
                    for (int o1 = 0; o1 < 2; ++o1)
                        for (int o2 = 0; o2 < 2; ++o2) {
                            if (T[o2][o1][0] && T[o2][o1][1]) g[0] += val[o2][o1][1] - val[o2][o1][0];
                            if (T[o2][0][o1] && T[o2][1][o1]) g[1] += val[o2][1][o1] - val[o2][0][o1];
                            if (T[0][o2][o1] && T[1][o2][o1]) g[2] += val[1][o2][o1] - val[0][o2][o1];
                        }
                    double r3[3];
                    for (int a3 = 0; a3 < 3; ++a3) r3[a3] = cnt[a3] ? 1.0 / cnt[a3] : 0.0;
                    const double h[3] = {g[0] * r3[0], g[1] * r3[1], g[2] * r3[2]};
                    const double iso = sT * nT;
                    double F[3];
                    F[0] = r3[0] * (iso * h[0] + dS * (M[0] * h[0] + M[3] * h[1] + M[4] * h[2]));
                    F[1] = r3[1] * (iso * h[1] + dS * (M[3] * h[0] + M[1] * h[1] + M[5] * h[2]));
                    F[2] = r3[2] * (iso * h[2] + dS * (M[4] * h[0] + M[5] * h[1] + M[2] * h[2]));
                    const int os = 1 - s, ot = 1 - t, ou = 1 - uu;
                    if (T[ou][ot][1 - os]) acc += (os ? 1.0 : -1.0) * F[0];
                    if (T[ou][1 - ot][os]) acc += (ot ? 1.0 : -1.0) * F[1];
                    if (T[1 - ou][ot][os]) acc += (ou ? 1.0 : -1.0) * F[2];
                }
        out[q] = (real)(C * acc);
    }
}

// ---------------------------------------------------------------------------
// Per-component reductions over the component-sorted tissue index list.
// One CTA per chunk; the last CTA forms every component's mean in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kChunk = 2048;

template <typename real>
__device__ __forceinline__ const real *pick_iterate(const real *x0, const real *x1, int by_parity, const Ctl *ctl)
{
    return (by_parity && (ctl->iters & 1)) ? x1 : x0;
}

// means[c] = mean over component c of x (x = x1 when by_parity and the finished
// solve took an odd number of sweeps).
template <typename real>
__global__ void __launch_bounds__(kRedThreads)
k_comp_mean(const real *x0, const real *x1, int by_parity, const int *idx, const Chunk *chunks,
            const int *comp_chunk0, const long long *comp_count, int ncomp, double *partials,
            double *means, Ctl *ctl)
{
    __shared__ double sred[kRedThreads / 32];
    __shared__ int sLast;
    const real *x = pick_iterate(x0, x1, by_parity, ctl);
    const Chunk ch = chunks[blockIdx.x];
    double s = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) s += (double)x[idx[i]];
    s = block_sum<kRedThreads>(s, sred);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        sLast = (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    for (int c = threadIdx.x; c < ncomp; c += kRedThreads) {
        double t = 0.0;
        for (int i = comp_chunk0[c]; i < comp_chunk0[c + 1]; ++i) t += ((volatile double *)partials)[i];
        means[c] = t / (double)comp_count[c];
    }
    if (threadIdx.x == 0) ctl->arrive = 0;
}

// x <- x - means[comp] on the tissue.  With want_norm the last CTA also forms
// ||x||^2 (after the correction) and starts a new elliptic solve in ctl.
template <typename real>
__global__ void __launch_bounds__(kRedThreads)
k_comp_subtract(real *x, const int *idx, const Chunk *chunks, const double *means, int want_norm,
                double rel_tol2, double *partials, Ctl *ctl)
{
    __shared__ double sred[kRedThreads / 32];
    __shared__ int sLast;
    const Chunk ch = chunks[blockIdx.x];
    const double m = means[ch.comp];
    double s = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = idx[i];
        const real v = (real)((double)x[q] - m);
        x[q] = v;
        s += (double)v * (double)v;
    }
    if (!want_norm) return;
    s = block_sum<kRedThreads>(s, sred);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        sLast = (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!sLast) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kRedThreads) t += ((volatile double *)partials)[i];
    t = block_sum<kRedThreads>(t, sred);
    if (threadIdx.x == 0) {
        ctl->arrive = 0;
        ctl->bnorm2 = t;
        ctl->thresh2 = rel_tol2 * t;
        ctl->sweep = 0;
        ctl->iters = 0;
        ctl->converged = (t == 0.0);
        ctl->diverged = 0;
        ctl->rnorm2 = 0.0;
        ctl->done = (t == 0.0) || !(t == t) || isinf(t);
        if (!(t == t) || isinf(t)) ctl->nonfinite = 1;
        __threadfence();
    }
}

// ve <- x_final - means[comp]; x_final is x1 when the solve took an odd number of sweeps.
template <typename real>
__global__ void __launch_bounds__(kRedThreads)
k_project(real *x0, const real *x1, const int *idx, const Chunk *chunks, const double *means, const Ctl *ctl)
{
    const real *src = (ctl->iters & 1) ? x1 : x0;
    const Chunk ch = chunks[blockIdx.x];
    const double m = means[ch.comp];
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = idx[i];
        x0[q] = (real)((double)src[q] - m);
    }
}

template <typename real>
__global__ void k_fill(real *p, long long n, real v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace gbep
