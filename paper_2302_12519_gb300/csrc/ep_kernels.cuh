// ep_kernels.cuh -- sm_103a kernels of the voxel electrophysiology step.
//
// Operator (Sec. "Operators / Laplacian", Sec. "Matrix-Free Assembly",
// Eq. ass3 with F = dx I, and the conductivity block S1 of Sec. "Diffusion"):
//   at every grid vertex p (corner of a 2x2x2 voxel block)
//     h_a   = mean over the valid a-pairs of the block of (u_hi - u_lo)
//             (a pair is valid when both voxels are tissue: no-flux mask)
//     S_p   = (1/8) sum over tissue voxels j of the block of Sigma_j,
//             Sigma_j = sT I + (sL - sT) f_j f_j^T                (Eq. sigma1)
//     Fh_a  = r_a (nT sT h + dS M h)_a,   r_a = 1 / (#valid a-pairs), 0 if none,
//             nT = #tissue voxels, M = sum f f^T, dS = sL - sT
//   at every tissue voxel q
//     (L u)_q = C * sum_a [ T(q - e_a) Phi_a^- - T(q + e_a) Phi_a^+ ],
//             Phi = sum of Fh_a over the 4 vertices of the face,
//             C = 1 / (8 dx^2).
//   L u approximates -div(Sigma grad u); L is symmetric PSD and conserves
//   charge (L 1 = 0).
//
// Work decomposition (the GB300 design, not the paper's one-thread-per-row):
// a CTA owns a 30 x kTileY column of output voxels and marches through a
// z-range ("segment").  Warp w handles the voxel rows (y0 + w - 1, y0 + w):
// lane l holds voxel column x0 - 1 + l, so x-neighbours come from warp
// shuffles and tissue flags of a whole row from one ballot.  Each warp
// computes the vertex row between its two voxel rows; the vertex row below
// is taken from warp w - 1 through shared memory (one barrier per z-plane).
// Values of the previous z-plane stay in registers, so every voxel is read
// from memory once per plane by each of the two warps that touch its row
// (the second read hits L1).  The fibre tensor sums are recomputed from fp16
// fibres on every pass instead of being stored, which keeps the traffic at
// one 8-byte record per voxel.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbep {

constexpr int kWarps = 8;                  // warps per CTA
constexpr int kThreads = kWarps * 32;
constexpr int kTileX = 30;                 // output voxels per row (lanes 1..30)
constexpr int kTileY = kWarps - 1;         // output rows per CTA (warps 1..kWarps-1)
constexpr int kMaxStim = 8;
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned short kNonTissue = 0xBC00u;  // fp16 -1.0: record lane 3 of a non-tissue voxel

enum Mode { M_APPLY = 0, M_RHS = 1, M_PAR_MONO = 2, M_PAR_BI = 3, M_JAC = 4 };

struct Seg {
    int bx, by, k0, k1;   // tile column and output planes [k0, k1)
};

struct StimBox {
    int lo[3], hi[3];
    double amp;
};

struct StimSet {
    int n;                // boxes active at this step
    StimBox box[kMaxStim];
};

// Device control block of the elliptic solve.
struct Ctl {
    unsigned int arrive;  // CTAs that finished the current launch (reset by the last one)
    int done;             // solve finished: converged, capped, diverged or empty rhs
    int sweep;            // sweeps done in the current solve
    int iters;            // sweeps of the finished solve
    int converged;
    int nonfinite;
    int diverged;
    int pad;
    double bnorm2;        // ||b||^2 after the mean correction
    double thresh2;       // rel_tol^2 * ||b||^2
    double rnorm2;        // ||r||^2 at the last check
};

struct Chunk {
    int start, end, comp;  // [start, end) into the component-sorted tissue index list
};

template <typename real>
struct StencilArgs {
    int nx, ny, nz;
    const Seg *segs;
    const ushort4 *rec;   // (fx, fy, fz, 1/Dhat) in fp16; lane 3 = -1 off the tissue
    const real *u;        // APPLY/RHS: operand; PAR: v (old)
    const real *w;        // PAR: w (old)
    const real *ve;       // PAR_BI: ve
    const real *b;        // JAC: right-hand side
    real *out;            // APPLY: L u; RHS: b; PAR: v (new)
    real *wout;           // PAR: w (new)
    real *tact;           // PAR: activation times
    real *x0, *x1;        // JAC: ping-pong iterates (x0 holds the warm start)
    real sT, dS, C;       // operator: sigma_T, sigma_L - sigma_T, 1/(8 dx^2)
    real coef;            // PAR: dt/K (times lambda/(1+lambda) for MONO); JAC: omega / C
    real dt, inv_tin, inv_tout, inv_topen, inv_tclose, vgate;
    double tn, dt_d;      // PAR: t_n and dt (activation time, double)
    StimSet stim;         // PAR: boxes active at t_n
    int check_every;      // JAC
    int max_iter;         // JAC
    double div_factor;    // JAC: stop as diverged when ||r||^2 > div_factor * ||b||^2
    double *partials;     // JAC: one per CTA
    Ctl *ctl;             // JAC
};

__device__ __forceinline__ float h2f(unsigned short b) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ bool rec_tissue(const ushort4 &r) { return (r.w & 0x8000u) == 0; }

template <typename real>
__device__ __forceinline__ real rcp_count(int n)
{
    return n == 1 ? real(1) : n == 2 ? real(0.5) : n == 3 ? real(1) / real(3) : n == 4 ? real(0.25) : real(0);
}

template <typename real>
__device__ __forceinline__ real shfl_up(real v) { return __shfl_up_sync(kFull, v, 1); }
template <typename real>
__device__ __forceinline__ real shfl_dn(real v) { return __shfl_down_sync(kFull, v, 1); }

// Mitchell-Schaeffer explicit Euler (Eqs. ms1, ms2; closing branch -w/tau_close).
template <typename real>
__device__ __forceinline__ void ms_step(const StencilArgs<real> &a, real v, real w, int x, int y, int z,
                                        real &vstar, real &wnew)
{
    real js = 0;
    for (int s = 0; s < a.stim.n; ++s) {
        const StimBox &bx = a.stim.box[s];
        if (x >= bx.lo[0] && x < bx.hi[0] && y >= bx.lo[1] && y < bx.hi[1] && z >= bx.lo[2] && z < bx.hi[2])
            js += real(bx.amp);
    }
    real jin = v * v * (real(1) - v) * w * a.inv_tin;
    real jout = -v * a.inv_tout;
    vstar = v + a.dt * (jin + jout + js);
    real dw = (v < a.vgate) ? (real(1) - w) * a.inv_topen : -w * a.inv_tclose;
    wnew = w + a.dt * dw;
}

// Fixed-order block reduction of one double per thread; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sred)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sred[wid] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NT / 32; ++i) s += sred[i];
    return s;
}

template <typename real, int MODE>
__global__ void __launch_bounds__(kThreads) k_stencil(StencilArgs<real> a)
{
    __shared__ real sF[2][3][kWarps][32];   // vertex fluxes, double-buffered by plane parity
    __shared__ unsigned sM[2][kWarps];      // tissue ballot of each warp's lower row
    __shared__ double sred[kWarps];
    __shared__ int sLast;

    int sweep = 0;
    bool check = false;
    const real *src = a.u;
    real *dst = a.out;
    if (MODE == M_JAC) {
        if (a.ctl->done) return;            // converged earlier: queued sweeps are no-ops
        sweep = a.ctl->sweep;
        src = (sweep & 1) ? a.x1 : a.x0;
        dst = (sweep & 1) ? a.x0 : a.x1;
        check = (sweep % a.check_every) == 0;
    }

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const Seg sg = a.segs[blockIdx.x];
    const int x = sg.bx * kTileX - 1 + lane;
    const int ylo = sg.by * kTileY + wid - 1;   // output row of this warp
    const int yhi = ylo + 1;
    const bool xin = x >= 0 && x < a.nx;
    const bool lo_in = xin && ylo >= 0 && ylo < a.ny;
    const bool hi_in = xin && yhi >= 0 && yhi < a.ny;
    const long long plane = (long long)a.nx * a.ny;
    const long long qlo0 = lo_in ? (long long)x + (long long)a.nx * ylo : 0;
    const long long qhi0 = hi_in ? (long long)x + (long long)a.nx * yhi : 0;
    const bool out_lane = lane >= 1 && lane <= kTileX && wid >= 1 && lo_in;
    const real sT = a.sT, dS = a.dS;

    // previous-plane registers
    real uLo_p = 0, uHi_p = 0, uLoL_p = 0, uHiL_p = 0;
    real P_p[6] = {0, 0, 0, 0, 0, 0};
    unsigned mLo_p = 0, mHi_p = 0, mLo_pp = 0, mYm_p = 0;
    real FB_p[3] = {0, 0, 0}, FA_p[3] = {0, 0, 0};
    // own output voxel of the previous plane
    real eA_p = 0, eB_p = 0, eC_p = 0;   // PAR: v*, w_new, v_old ; JAC: b, 1/Dhat, - ; others unused
    float acc = 0.f;                      // JAC: sum of r^2 (this thread's voxels)
    int par = 0;

    for (int k = sg.k0 - 1; k <= sg.k1; ++k) {
        const bool kin = k >= 0 && k < a.nz;
        real uLo = 0, uHi = 0;
        real fLo[3] = {0, 0, 0}, fHi[3] = {0, 0, 0};
        bool tLo = false, tHi = false;
        real eA = 0, eB = 0, eC = 0;
        // ---- load the two voxel rows of plane k ----
        if (kin && lo_in) {
            const long long q = qlo0 + (long long)k * plane;
            const ushort4 r = a.rec[q];
            if (rec_tissue(r)) {
                tLo = true;
                fLo[0] = h2f(r.x); fLo[1] = h2f(r.y); fLo[2] = h2f(r.z);
                if (MODE == M_APPLY || MODE == M_RHS) {
                    uLo = a.u[q];
                } else if (MODE == M_JAC) {
                    uLo = src[q];
                    eA = a.b[q];
                    eB = h2f(r.w);
                } else {
                    const real v = a.u[q], w = a.w[q];
                    real vs, wn;
                    ms_step(a, v, w, x, ylo, k, vs, wn);
                    uLo = (MODE == M_PAR_BI) ? vs + a.ve[q] : vs;
                    eA = vs; eB = wn; eC = v;
                }
            }
        }
        if (kin && hi_in) {
            const long long q = qhi0 + (long long)k * plane;
            const ushort4 r = a.rec[q];
            if (rec_tissue(r)) {
                tHi = true;
                fHi[0] = h2f(r.x); fHi[1] = h2f(r.y); fHi[2] = h2f(r.z);
                if (MODE == M_APPLY || MODE == M_RHS) {
                    uHi = a.u[q];
                } else if (MODE == M_JAC) {
                    uHi = src[q];
                } else {
                    const real v = a.u[q], w = a.w[q];
                    real vs, wn;
                    ms_step(a, v, w, x, yhi, k, vs, wn);
                    uHi = (MODE == M_PAR_BI) ? vs + a.ve[q] : vs;
                }
            }
        }
        const unsigned mLo = __ballot_sync(kFull, tLo), mHi = __ballot_sync(kFull, tHi);
        const real uLoL = shfl_up(uLo), uHiL = shfl_up(uHi);
        // own-column tensor sum of this plane: fLo fLo^T + fHi fHi^T (zero fibres off tissue)
        real P[6];
        P[0] = fLo[0] * fLo[0] + fHi[0] * fHi[0];
        P[1] = fLo[1] * fLo[1] + fHi[1] * fHi[1];
        P[2] = fLo[2] * fLo[2] + fHi[2] * fHi[2];
        P[3] = fLo[0] * fLo[1] + fHi[0] * fHi[1];
        P[4] = fLo[0] * fLo[2] + fHi[0] * fHi[2];
        P[5] = fLo[1] * fLo[2] + fHi[1] * fHi[2];

        if (k >= sg.k0) {
            // ---- vertex (x - 1/2, yhi - 1/2, k - 1/2): block columns L = x-1, O = x ----
            const unsigned bO = 1u << lane;
            const unsigned bL = lane ? (1u << (lane - 1)) : 0u;
            const bool Olc = mLo & bO, Ohc = mHi & bO, Olp = mLo_p & bO, Ohp = mHi_p & bO;
            const bool Llc = mLo & bL, Lhc = mHi & bL, Llp = mLo_p & bL, Lhp = mHi_p & bL;
            int nx_ = 0, ny_ = 0, nz_ = 0;
            real gx = 0, gy = 0, gz = 0;
            // x-pairs (L, O) in rows lo/hi, planes p/c
            if (Llp && Olp) { gx += uLo_p - uLoL_p; ++nx_; }
            if (Lhp && Ohp) { gx += uHi_p - uHiL_p; ++nx_; }
            if (Llc && Olc) { gx += uLo - uLoL; ++nx_; }
            if (Lhc && Ohc) { gx += uHi - uHiL; ++nx_; }
            // y-pairs (lo, hi) in columns L/O, planes p/c
            if (Olp && Ohp) { gy += uHi_p - uLo_p; ++ny_; }
            if (Llp && Lhp) { gy += uHiL_p - uLoL_p; ++ny_; }
            if (Olc && Ohc) { gy += uHi - uLo; ++ny_; }
            if (Llc && Lhc) { gy += uHiL - uLoL; ++ny_; }
            // z-pairs (p, c) in columns L/O, rows lo/hi
            if (Olp && Olc) { gz += uLo - uLo_p; ++nz_; }
            if (Ohp && Ohc) { gz += uHi - uHi_p; ++nz_; }
            if (Llp && Llc) { gz += uLoL - uLoL_p; ++nz_; }
            if (Lhp && Lhc) { gz += uHiL - uHiL_p; ++nz_; }
            const int nT = (int)Olc + Ohc + Olp + Ohp + Llc + Lhc + Llp + Lhp;
            real Q[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) Q[i] = P[i] + P_p[i];
            real M[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) M[i] = Q[i] + shfl_up(Q[i]);
            const real rx = rcp_count<real>(nx_), ry = rcp_count<real>(ny_), rz = rcp_count<real>(nz_);
            const real hx = gx * rx, hy = gy * ry, hz = gz * rz;
            const real iso = sT * real(nT);
            real FB[3];
            FB[0] = rx * (iso * hx + dS * (M[0] * hx + M[3] * hy + M[4] * hz));
            FB[1] = ry * (iso * hy + dS * (M[3] * hx + M[1] * hy + M[5] * hz));
            FB[2] = rz * (iso * hz + dS * (M[4] * hx + M[5] * hy + M[2] * hz));
            // ---- exchange vertex rows between warps ----
            sF[par][0][wid][lane] = FB[0];
            sF[par][1][wid][lane] = FB[1];
            sF[par][2][wid][lane] = FB[2];
            if (lane == 0) sM[par][wid] = mLo;
            __syncthreads();
            real FA[3] = {0, 0, 0};
            unsigned mYm = 0;
            if (wid >= 1) {
                FA[0] = sF[par][0][wid - 1][lane];
                FA[1] = sF[par][1][wid - 1][lane];
                FA[2] = sF[par][2][wid - 1][lane];
                mYm = sM[par][wid - 1];
            }
            par ^= 1;

            if (k >= sg.k0 + 1) {
                // ---- output voxel (x, ylo, k - 1) ----
                const real phxm = FA_p[0] + FA[0] + FB_p[0] + FB[0];
                const real phxp = shfl_dn(phxm);
                const real psyA = FA_p[1] + FA[1];
                const real phym = psyA + shfl_dn(psyA);
                const real psyB = FB_p[1] + FB[1];
                const real phyp = psyB + shfl_dn(psyB);
                const real pszP = FA_p[2] + FB_p[2];
                const real phzm = pszP + shfl_dn(pszP);
                const real pszC = FA[2] + FB[2];
                const real phzp = pszC + shfl_dn(pszC);
                const bool self = mLo_p & bO;
                if (out_lane && self) {
                    real s = 0;
                    if (mLo_p & bL) s += phxm;
                    if (mLo_p & (bO << 1)) s -= phxp;
                    if (mYm_p & bO) s += phym;
                    if (mHi_p & bO) s -= phyp;
                    if (mLo_pp & bO) s += phzm;
                    if (mLo & bO) s -= phzp;
                    const real Lu = a.C * s;
                    const long long q = qlo0 + (long long)(k - 1) * plane;
                    if (MODE == M_APPLY) {
                        a.out[q] = Lu;
                    } else if (MODE == M_RHS) {
                        a.out[q] = -Lu;
                    } else if (MODE == M_JAC) {
                        const real r = eA_p - Lu;
                        dst[q] = uLo_p + a.coef * eB_p * r;
                        if (check) acc += (float)r * (float)r;
                    } else {
                        const real vnew = eA_p - a.coef * Lu;
                        a.out[q] = vnew;
                        a.wout[q] = eB_p;
                        const real vold = eC_p;
                        if (vold < real(0.5) && vnew >= real(0.5)) {
                            const real t0 = a.tact[q];
                            if (t0 < real(0))
                                a.tact[q] = (real)(a.tn + a.dt_d * (0.5 - (double)vold) / ((double)vnew - (double)vold));
                        }
                        if (!isfinite((double)vnew)) atomicOr(&a.ctl->nonfinite, 1);
                    }
                }
            }
            FA_p[0] = FA[0]; FA_p[1] = FA[1]; FA_p[2] = FA[2];
            FB_p[0] = FB[0]; FB_p[1] = FB[1]; FB_p[2] = FB[2];
            mYm_p = mYm;
        }
        // ---- rotate plane registers ----
        uLo_p = uLo; uHi_p = uHi; uLoL_p = uLoL; uHiL_p = uHiL;
#pragma unroll
        for (int i = 0; i < 6; ++i) P_p[i] = P[i];
        mLo_pp = mLo_p; mLo_p = mLo; mHi_p = mHi;
        eA_p = eA; eB_p = eB; eC_p = eC;
    }

    if (MODE == M_JAC) {
        // residual norm of this sweep's input: per-thread FP32 partial over its
        // few voxels, FP64 above; deterministic fixed-order reduction
        double tot = block_sum<kThreads>(check ? (double)acc : 0.0, sred);
        if (threadIdx.x == 0) {
            a.partials[blockIdx.x] = tot;
            __threadfence();
            sLast = (atomicAdd(&a.ctl->arrive, 1u) == gridDim.x - 1);
        }
        __syncthreads();
        if (sLast) {
            __threadfence();
            double s = 0;
            if (check)
                for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) s += ((volatile double *)a.partials)[i];
            s = block_sum<kThreads>(s, sred);
            if (threadIdx.x == 0) {
                Ctl *c = a.ctl;
                c->arrive = 0;
                const int j = sweep + 1;
                c->sweep = j;
                if (check) {
                    c->rnorm2 = s;
                    if (!(s == s) || isinf(s)) {
                        c->nonfinite = 1; c->done = 1; c->iters = j;
                    } else if (s <= c->thresh2) {
                        c->converged = 1; c->done = 1; c->iters = j;
                    } else if (s > a.div_factor * c->bnorm2) {
                        c->diverged = 1; c->done = 1; c->iters = j;
                    }
                }
                if (!c->done && j >= a.max_iter) { c->done = 1; c->iters = j; }
                __threadfence();
            }
        }
    }
}

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
