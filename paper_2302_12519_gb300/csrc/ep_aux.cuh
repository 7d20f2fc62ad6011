// ep_aux.cuh -- set-up, diagnostic and reduction kernels of the voxel electrophysiology step.
#pragma once

#include "ep_common.cuh"

namespace gbep {

// ---------------------------------------------------------------------------
// Setup and diagnostic kernels: one thread per voxel, vertices recomputed
// from global memory (8x redundant, used once at setup or for checking).
// ---------------------------------------------------------------------------

// Static data of vertex (I, J, K): tissue flags T, valid tissue-pair counts,
// nT and M = sum f f^T over the tissue voxels; with torso records also the
// domain flags Td (tissue or torso), domain-pair counts cntd and the torso
// voxel count nB.
__device__ inline void vertex_static(int nx, int ny, int nz, const float4 *rec, int I, int J, int K,
                                     int cnt[3], int &nT, double M[6], bool T[2][2][2], int cntd[3], int &nB,
                                     bool Td[2][2][2])
{
    double f[2][2][2][3];
    for (int u = 0; u < 2; ++u)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s) {
                const int i = I - 1 + s, j = J - 1 + t, k = K - 1 + u;
                bool in = i >= 0 && j >= 0 && k >= 0 && i < nx && j < ny && k < nz;
                T[u][t][s] = Td[u][t][s] = false;
                f[u][t][s][0] = f[u][t][s][1] = f[u][t][s][2] = 0.0;
                if (in) {
                    const float4 r = rec[(long long)i + (long long)nx * ((long long)j + (long long)ny * k)];
                    if (rec_tissue(r)) {
                        Td[u][t][s] = true;
                        T[u][t][s] = !rec_bath(r);
                        f[u][t][s][0] = r.x; f[u][t][s][1] = r.y; f[u][t][s][2] = r.z;
                    }
                }
            }
    nT = nB = 0;
    for (int i = 0; i < 6; ++i) M[i] = 0.0;
    cnt[0] = cnt[1] = cnt[2] = cntd[0] = cntd[1] = cntd[2] = 0;
    for (int u = 0; u < 2; ++u)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s) {
                if (Td[u][t][s] && !T[u][t][s]) ++nB;
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
            cntd[0] += Td[o2][o1][0] && Td[o2][o1][1];
            cntd[1] += Td[o2][0][o1] && Td[o2][1][o1];
            cntd[2] += Td[0][o2][o1] && Td[1][o2][o1];
        }
}

// The fp32 record of every voxel: the caller's fibre (fx, fy, fz) on the tissue,
// lane 3 filled by k_build_diag, -1 there off the records' domain.  With a torso
// (nullable), its voxels outside the tissue get the record (-0, 0, 0, .): in the
// domain, zero fibre, tagged; a tissue fibre lane 0 of -0 is stored as +0 so that
// the tag stays unique.
__global__ void k_build_records(int nx, int ny, int nz, const float *fib, const uint8_t *mask,
                                const uint8_t *torso, float4 *rec)
{
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        float4 r;
        if (mask[q]) {
            r.x = fib[3 * q + 0];
            r.y = fib[3 * q + 1];
            r.z = fib[3 * q + 2];
            if (__float_as_uint(r.x) == kBathTag) r.x = 0.0f;
            r.w = 0.0f;   // 1/Dhat filled by k_build_diag
        } else if (torso && torso[q]) {
            r.x = __uint_as_float(kBathTag);
            r.y = r.z = 0.0f;
            r.w = 0.0f;
        } else {
            r.x = r.y = r.z = 0.0f;
            r.w = kNonTissueW;
        }
        rec[q] = r;
    }
}

// Dhat_q = sum over the 8 vertices of q of c^T Shat c, c_a = +-T(partner) r_a,
// Shat = nT sT I + dS M; D_q = Dhat_q / (8 dx^2).
// Dhat of voxel (i, j, k) for the operator with sigma_T = sT and
// sigma_L - sigma_T = dS (tissue term, tissue voxels), plus with so > 0 the
// torso term so nB I over domain pairs (torso records): the diagonal of L is
// C Dhat, C = 1 / (8 dx^2).
__device__ inline double diag_hat(int nx, int ny, int nz, const float4 *rec, int i, int j, int k, double sT,
                                  double dS, double so)
{
    double D = 0.0;
    for (int u = 0; u < 2; ++u)
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < 2; ++s) {
                int cnt[3], cntd[3], nT, nB;
                double M[6];
                bool T[2][2][2], Td[2][2][2];
                vertex_static(nx, ny, nz, rec, i + s, j + t, k + u, cnt, nT, M, T, cntd, nB, Td);
                // q sits at block offset (1-s, 1-t, 1-u); partner along a flips that offset
                const int os = 1 - s, ot = 1 - t, ou = 1 - u;
                if (T[ou][ot][os]) {
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
                if (so > 0.0 && nB > 0) {
                    double c2 = 0.0;
                    if (Td[ou][ot][1 - os] && cntd[0]) c2 += 1.0 / ((double)cntd[0] * cntd[0]);
                    if (Td[ou][1 - ot][os] && cntd[1]) c2 += 1.0 / ((double)cntd[1] * cntd[1]);
                    if (Td[1 - ou][ot][os] && cntd[2]) c2 += 1.0 / ((double)cntd[2] * cntd[2]);
                    D += so * nB * c2;
                }
            }
    return D;
}

__global__ void k_build_diag(int nx, int ny, int nz, double sT, double dS, double so, const float4 *rec,
                             float4 *rec_out)
{
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        float4 r = rec[q];
        if (!rec_tissue(r)) { rec_out[q] = r; continue; }
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
        const double D = diag_hat(nx, ny, nz, rec, i, j, k, sT, dS, so);
        r.w = D > 0.0 ? (float)(1.0 / D) : 0.0f;
        rec_out[q] = r;
    }
}

// Implicit-Euler Jacobi (Eq. iejac1): inv_q = 1 / (1 + a C Dhat_q) for the
// intracellular operator on the tissue, 0 elsewhere.
template <typename real>
__global__ void k_build_ie_diag(int nx, int ny, int nz, double sT, double dS, double aC, const float4 *rec,
                                real *inv)
{
    const long long n = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        if (!rec_tissue(rec[q])) { inv[q] = real(0); continue; }
        const int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long long)nx * ny));
        inv[q] = (real)(1.0 / (1.0 + aC * diag_hat(nx, ny, nz, rec, i, j, k, sT, dS, 0.0)));
    }
}

// ---------------------------------------------------------------------------
// Per-component reductions over the component-sorted tissue index list.
// One work item per chunk (2048 tissue voxels of one component); the item
// that completes the launch for an instance finishes that instance in a fixed
// order, so results do not depend on scheduling.
// ---------------------------------------------------------------------------
struct RedSmem {
    double sred[kRedThreads / 32];
    int sflag;
};

enum RedField { RED_B = 0, RED_X_FINAL = 1 };

// Final iterate of an elliptic solve of `iters` sweeps at voxel q: x1 after an
// odd number of sweeps, else x0; in the correction form x0 + e, e the last
// correction (x1 after an odd number of sweeps, else x2; none after 0); x0 for
// the eight-colour sweep, which works in place.
template <typename real>
__device__ __forceinline__ double final_iterate(const Inst<real> &I, int iters, int q)
{
    if (I.solver == 2) return (double)I.x0[q];
    if (I.eform) {
        double x = (double)I.x0[q];
        if (iters > 0) x += (double)((iters & 1) ? I.x1[q] : I.x2[q]);
        return x;
    }
    return (double)((iters & 1) ? I.x1[q] : I.x0[q]);
}

// means[c] = mean over component c of b, or of the final iterate of the solve.
template <typename real>
__device__ __forceinline__ void comp_mean_item(const Inst<real> &I, int field, int item, int nitems, RedSmem &sm)
{
    Ctl *ctl = I.ctl;
    const int iters = ctl->iters;
    const Chunk ch = I.chunks[item];
    const bool rhs_torso = field == RED_B && I.torso;   // b is 0 on the torso (stale values there are skipped)
    double s = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = I.idx[i];
        if (field == RED_B) {
            if (!rhs_torso || rec_tissue(I.rec[q])) s += (double)I.b[q];
        } else {
            s += final_iterate(I, iters, q);
        }
    }
    s = block_sum<kRedThreads>(s, sm.sred);
    if (threadIdx.x == 0) I.partials[item] = s;
    if (!arrive_last(ctl, nitems, &sm.sflag)) return;
    for (int c = threadIdx.x; c < I.ncomp; c += kRedThreads) {
        double t = 0.0;
        for (int i = I.comp_chunk0[c]; i < I.comp_chunk0[c + 1]; ++i) t += ((volatile double *)I.partials)[i];
        I.means[c] = t / (double)I.comp_count[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->arrive = 0;
        __threadfence();
    }
}

// b <- b - means[comp] on the domain (with a torso, b counts as 0 on its voxels:
// the right-hand side -L_i v lives on the tissue); the item that completes the launch forms
// ||b||^2 and starts a new elliptic solve in the control block.
template <typename real>
__device__ __forceinline__ void comp_subtract_item(const Inst<real> &I, int item, int nitems, RedSmem &sm)
{
    Ctl *ctl = I.ctl;
    const Chunk ch = I.chunks[item];
    const double m = I.means[ch.comp];
    double s = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = I.idx[i];
        const double bq = (I.torso && !rec_tissue(I.rec[q])) ? 0.0 : (double)I.b[q];   // 0 on the torso
        const real v = (real)(bq - m);
        I.b[q] = v;
        s += (double)v * (double)v;
    }
    s = block_sum<kRedThreads>(s, sm.sred);
    if (threadIdx.x == 0) I.partials[item] = s;
    if (!arrive_last(ctl, nitems, &sm.sflag)) return;
    double t = 0.0;
    for (int i = threadIdx.x; i < nitems; i += kRedThreads) t += ((volatile double *)I.partials)[i];
    t = block_sum<kRedThreads>(t, sm.sred);
    if (threadIdx.x == 0) {
        ctl->arrive = 0;
        ctl->bnorm2 = t;
        ctl->thresh2 = I.rel_tol2 * t;
        ctl->sweep = 0;
        ctl->jarrive = 0;
        ctl->iters = 0;
        ctl->cycle0 = 0;
        ctl->r0n2 = 0.0;
        ctl->converged = (t == 0.0);
        ctl->diverged = 0;
        ctl->rnorm2 = 0.0;
        ctl->done = (t == 0.0) || !(t == t) || isinf(t);
        if (!(t == t) || isinf(t)) ctl->nonfinite = 1;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// Implicit-Euler diffusion (Sec. "Implicit Euler", Eq. iejac1).
// ---------------------------------------------------------------------------

// Monodomain: the reaction alone, one thread per tissue voxel of the list:
// f = v* (right-hand side, in b), first iterate v* (in the new v buffer), w+.
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_ie_react(Inst<real> I)
{
    const long long step = I.ctl->step;
    const int cur = (int)(step & 1);
    const double tn = (double)step * I.dt_d;
    const real *v = I.v[cur], *w = I.w[cur];
    real *vn = I.v[cur ^ 1], *wn = I.w[cur ^ 1];
    const long long nt = (long long)I.chunks[I.nchunk - 1].end;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nt; i += (long long)gridDim.x * blockDim.x) {
        const int q = I.idx[i];
        const int x = q % I.nx, y = (q / I.nx) % I.ny, z = q / (I.nx * I.ny);
        real vs, ws;
        ms_step(I, tn, v[q], w[q], x, y, z, vs, ws);
        I.b[q] = vs;
        vn[q] = vs;
        wn[q] = ws;
    }
}

// Start of an implicit solve: ||f||^2 over the tissue chunks (FP64, fixed
// order); the item that completes the launch resets the solve in the
// control block.
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_ie_start(Inst<real> I)
{
    __shared__ RedSmem sm;
    Ctl *ctl = I.ctl;
    const Chunk ch = I.chunks[blockIdx.x];
    double s = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const double f = (double)I.b[I.idx[i]];
        s += f * f;
    }
    s = block_sum<kRedThreads>(s, sm.sred);
    if (threadIdx.x == 0) I.partials[blockIdx.x] = s;
    if (!arrive_last(ctl, gridDim.x, &sm.sflag)) return;
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kRedThreads) t += ((volatile double *)I.partials)[i];
    t = block_sum<kRedThreads>(t, sm.sred);
    if (threadIdx.x == 0) {
        ctl->arrive = 0;
        ctl->bnorm2 = t;
        ctl->thresh2 = I.rel_tol2 * t;
        ctl->sweep = 0;
        ctl->jarrive = 0;
        ctl->iters = 0;
        ctl->cycle0 = 0;
        ctl->r0n2 = 0.0;
        ctl->converged = (t == 0.0);
        ctl->diverged = 0;
        ctl->rnorm2 = 0.0;
        ctl->done = (t == 0.0) || !(t == t) || isinf(t);
        if (!(t == t) || isinf(t)) ctl->nonfinite = 1;
        __threadfence();
    }
}

// End of an implicit solve: the final iterate (in ie_x after an odd number of
// sweeps) becomes v of the new step; activation times (first upward crossing
// of 0.5, linear in t) and the non-finite flag as in the explicit step.
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_ie_finish(Inst<real> I)
{
    Ctl *ctl = I.ctl;
    const long long step = ctl->step;
    const int cur = (int)(step & 1);
    const int iters = ctl->iters;
    const double tn = (double)step * I.dt_d;
    const real *vold = I.v[cur];
    real *vnew = I.v[cur ^ 1];
    const long long nt = (long long)I.chunks[I.nchunk - 1].end;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nt; i += (long long)gridDim.x * blockDim.x) {
        const int q = I.idx[i];
        const real v1 = (iters & 1) ? I.ie_x[q] : vnew[q];
        if (iters & 1) vnew[q] = v1;
        const real v0 = vold[q];
        if (v0 < real(0.5) && v1 >= real(0.5) && I.tact[q] < real(0))
            I.tact[q] = (real)(tn + I.dt_d * (0.5 - (double)v0) / ((double)v1 - (double)v0));
        if (!isfinite((double)v1)) atomicOr(&ctl->nonfinite, 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->ie_total += iters;
}

// ---------------------------------------------------------------------------
// Lanczos process for the spectrum of D^-1 A (Chebyshev interval at set-up),
// in the D inner product <x, y> = sum D x y, where D^-1 A is self-adjoint;
// D_q = C / (1/Dhat_q) from the fp32 record, voxels with an empty row left
// out.  One CTA per tissue chunk; FP64 partials (two per chunk in k_lz_proj);
// the item that completes a launch finishes it.  Scalars: lz[0] alpha, lz[1] beta of the current step,
// lz[2 + 2j] alpha_j, lz[3 + 2j] beta_{j+1}.
// ---------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ double lz_diag(const Inst<real> &I, int q)
{
    const float h = I.rec[q].w;
    return h > 0.0f ? (double)I.C / (double)h : 0.0;
}

// w = D^-1 t - beta vprev (t = A v); alpha = <w, v>_D
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_lz_w(Inst<real> I, const real *t, const real *v, const real *vprev,
                                                     real *w, double *lz)
{
    __shared__ RedSmem sm;
    const Chunk ch = I.chunks[blockIdx.x];
    const double beta = lz[1];
    double sa = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = I.idx[i];
        const double d = lz_diag(I, q);
        const double wq = d > 0.0 ? (double)t[q] / d - beta * (double)vprev[q] : 0.0;
        w[q] = (real)wq;
        sa += d * wq * (double)v[q];
    }
    sa = block_sum<kRedThreads>(sa, sm.sred);
    if (threadIdx.x == 0) I.partials[blockIdx.x] = sa;
    if (!arrive_last(I.ctl, gridDim.x, &sm.sflag)) return;
    double tsum = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kRedThreads) tsum += ((volatile double *)I.partials)[i];
    tsum = block_sum<kRedThreads>(tsum, sm.sred);
    if (threadIdx.x == 0) {
        I.ctl->arrive = 0;
        lz[0] = tsum;
        __threadfence();
    }
}

// w -= alpha v; per component the D-weighted mean of w (the null-space
// coefficient: the constants of each component span the null space) into means[c]
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_lz_proj(Inst<real> I, const real *v, real *w, const double *lz,
                                                        int use_alpha)
{
    __shared__ RedSmem sm;
    const Chunk ch = I.chunks[blockIdx.x];
    const double alpha = use_alpha ? lz[0] : 0.0;
    double sn = 0.0, sd = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = I.idx[i];
        const double d = lz_diag(I, q);
        const double wq = (double)w[q] - alpha * (double)v[q];
        w[q] = (real)wq;
        sn += d * wq;
        sd += d;
    }
    sn = block_sum<kRedThreads>(sn, sm.sred);
    const double dsum = block_sum<kRedThreads>(sd, sm.sred);
    if (threadIdx.x == 0) {
        I.partials[2 * blockIdx.x] = sn;
        I.partials[2 * blockIdx.x + 1] = dsum;
    }
    if (!arrive_last(I.ctl, gridDim.x, &sm.sflag)) return;
    for (int c = threadIdx.x; c < I.ncomp; c += kRedThreads) {
        double tn = 0.0, td = 0.0;
        for (int i = I.comp_chunk0[c]; i < I.comp_chunk0[c + 1]; ++i) {
            tn += ((volatile double *)I.partials)[2 * i];
            td += ((volatile double *)I.partials)[2 * i + 1];
        }
        I.means[c] = td > 0.0 ? tn / td : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        I.ctl->arrive = 0;
        __threadfence();
    }
}

// w -= means[comp] on the coupled voxels; beta' = ||w||_D; records alpha_j, beta_{j+1}
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_lz_norm(Inst<real> I, real *w, double *lz, int j)
{
    __shared__ RedSmem sm;
    const Chunk ch = I.chunks[blockIdx.x];
    const double m = I.means[ch.comp];
    double s2 = 0.0;
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = I.idx[i];
        const double d = lz_diag(I, q);
        const double wq = d > 0.0 ? (double)w[q] - m : 0.0;
        w[q] = (real)wq;
        s2 += d * wq * wq;
    }
    s2 = block_sum<kRedThreads>(s2, sm.sred);
    if (threadIdx.x == 0) I.partials[blockIdx.x] = s2;
    if (!arrive_last(I.ctl, gridDim.x, &sm.sflag)) return;
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kRedThreads) t += ((volatile double *)I.partials)[i];
    t = block_sum<kRedThreads>(t, sm.sred);
    if (threadIdx.x == 0) {
        I.ctl->arrive = 0;
        lz[1] = sqrt(t);
        if (j >= 0) {
            lz[2 + 2 * j] = lz[0];
            lz[3 + 2 * j] = lz[1];
        }
        __threadfence();
    }
}

// vprev = v; v = w / beta (the next Lanczos vector)
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_lz_next(Inst<real> I, long long nt, real *v, real *vprev,
                                                        const real *w, const double *lz)
{
    const double inv = lz[1] > 0.0 ? 1.0 / lz[1] : 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nt; i += (long long)gridDim.x * blockDim.x) {
        const int q = I.idx[i];
        vprev[q] = v[q];
        v[q] = (real)((double)w[q] * inv);
    }
}

// Start vector on the coupled tissue voxels: splitmix64 of the voxel index,
// uniform in [-1/2, 1/2).
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_lz_start(Inst<real> I, long long nt, real *w)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nt; i += (long long)gridDim.x * blockDim.x) {
        const int q = I.idx[i];
        unsigned long long z = 0x9E3779B97F4A7C15ull * (unsigned long long)(q + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        w[q] = lz_diag(I, q) > 0.0 ? (real)((double)(z >> 11) * 0x1.0p-53 - 0.5) : real(0);
    }
}

// ECG (Sec. "Electrocardiogram"): the potentials at the three electrode voxels
// (RA, LA, LL) after the solve, appended to the record as sample `slot`.
template <typename real>
__global__ void k_ecg_record(const real *ve, int q0, int q1, int q2, double *rec, long long slot)
{
    const int t = threadIdx.x;
    if (t < 3) rec[3 * slot + t] = (double)ve[t == 0 ? q0 : (t == 1 ? q1 : q2)];
}

// v_e <- x_final - means[comp] (written to x0, the warm start of the next solve).
template <typename real>
__device__ __forceinline__ void project_item(const Inst<real> &I, int item)
{
    const int iters = I.ctl->iters;
    const Chunk ch = I.chunks[item];
    const double m = I.means[ch.comp];
    for (int i = ch.start + threadIdx.x; i < ch.end; i += kRedThreads) {
        const int q = I.idx[i];
        I.x0[q] = (real)(final_iterate(I, iters, q) - m);
    }
}

template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_comp_mean(Inst<real> I, int field)
{
    __shared__ RedSmem sm;
    comp_mean_item(I, field, blockIdx.x, gridDim.x, sm);
}

template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_comp_subtract(Inst<real> I)
{
    __shared__ RedSmem sm;
    comp_subtract_item(I, blockIdx.x, gridDim.x, sm);
}

template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_project(Inst<real> I)
{
    project_item(I, blockIdx.x);
}

// Batched forms: one persistent launch over the packed (instance, chunk) list.
template <typename real>
__global__ void __launch_bounds__(kRedThreads)
k_comp_mean_batch(const Inst<real> *insts, const BItem *items, int nitems, int field)
{
    __shared__ RedSmem sm;
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BItem it = items[i];
        comp_mean_item(insts[it.inst], field, it.item, it.nitems, sm);
        __syncthreads();
    }
}

template <typename real>
__global__ void __launch_bounds__(kRedThreads)
k_comp_subtract_batch(const Inst<real> *insts, const BItem *items, int nitems)
{
    __shared__ RedSmem sm;
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BItem it = items[i];
        comp_subtract_item(insts[it.inst], it.item, it.nitems, sm);
        __syncthreads();
    }
}

template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_project_batch(const Inst<real> *insts, const BItem *items, int nitems)
{
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
        const BItem it = items[i];
        project_item(insts[it.inst], it.item);
    }
}

// ---------------------------------------------------------------------------
// Step control (single thread per instance).
// ---------------------------------------------------------------------------

// End of a step: the step counter moves on (v, w of the new step are in buffer
// (step + 1) & 1 already); the solve's sweeps are added to the total.
template <typename real>
__global__ void k_end_step(const Inst<real> *insts, int ninst, Inst<real> one)
{
    for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < (insts ? ninst : 1); i += blockDim.x * gridDim.x) {
        Ctl *c = insts ? insts[i].ctl : one.ctl;
        const int model = insts ? insts[i].model : one.model;
        if (model == MODEL_BI) c->total_iters += c->iters;
        c->step += 1;
    }
}

template <typename real>
__global__ void k_fill(real *p, long long n, real v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Members of rows [0, n) swept by the packed kernel (packed[i] != 0) whose
// solve is unfinished, in row order: act[k] = {items before member k, its
// row, its control block}; entries n_active .. n hold {total items, -1,
// null}, so the rest of the list never matches an item; counts = {total
// items, n_active}.  Sets the condition of the device-side convergence loop:
// any member of rows [0, n) still active, packed or not.  One CTA of
// kActThreads.
constexpr int kActThreads = 1024;

template <typename real>
__global__ void __launch_bounds__(kActThreads)
k_active_list(const Inst<real> *insts, const int *packed, int n, ActRec *act, int *counts,
              cudaGraphConditionalHandle h)
{
    __shared__ int swa[32], swc[32];
    __shared__ int base_a, base_c;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base_a = base_c = 0;
    __syncthreads();
    int running = 0;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        int a = 0, c = 0;
        Ctl *ctl = i < n ? insts[i].ctl : nullptr;
        const bool live = i < n && !*(volatile int *)&ctl->done;
        running |= live ? 1 : 0;
        if (live && packed[i]) {
            a = 1;
            c = insts[i].nseg;
        }
        int sa = a, sc = c;   // inclusive scans within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const int ta = __shfl_up_sync(kFull, sa, o), tc = __shfl_up_sync(kFull, sc, o);
            if (lane >= o) {
                sa += ta;
                sc += tc;
            }
        }
        if (lane == 31) {
            swa[wid] = sa;
            swc[wid] = sc;
        }
        __syncthreads();
        if (wid == 0) {   // inclusive scan of the warp totals
            int va = lane < nw ? swa[lane] : 0, vc = lane < nw ? swc[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int ta = __shfl_up_sync(kFull, va, o), tc = __shfl_up_sync(kFull, vc, o);
                if (lane >= o) {
                    va += ta;
                    vc += tc;
                }
            }
            if (lane < nw) {
                swa[lane] = va;
                swc[lane] = vc;
            }
        }
        __syncthreads();
        if (a) {
            const int pa = base_a + (wid ? swa[wid - 1] : 0) + sa - a;
            act[pa] = ActRec{base_c + (wid ? swc[wid - 1] : 0) + sc - c, i, ctl};
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            base_a += swa[nw - 1];
            base_c += swc[nw - 1];
        }
        __syncthreads();
    }
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) {
        counts[0] = base_c;
        counts[1] = base_a;
        if (h) cudaGraphSetConditional(h, running ? 1u : 0u);
    }
    __syncthreads();
    for (int k = base_a + threadIdx.x; k <= n; k += blockDim.x) act[k] = ActRec{base_c, -1, nullptr};
}

// Outer loop of a multi-step graph: counts down the steps left in the chunk.
__global__ void k_steps_cond(long long *steps_left, cudaGraphConditionalHandle h)
{
    const long long left = *steps_left - 1;
    *steps_left = left;
    cudaGraphSetConditional(h, left > 0 ? 1u : 0u);
}

}  // namespace gbep
