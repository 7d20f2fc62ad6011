// ep_common.cuh -- shared definitions of the sm_103a kernels of the voxel
// electrophysiology step (work items, control block, kernel arguments, the
// Mitchell-Schaeffer update and a fixed-order block reduction).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbep {

#ifndef EP_WARPS
#define EP_WARPS 8
#endif
#ifndef EP_MIN_BLOCKS
#define EP_MIN_BLOCKS 3
#endif
constexpr int kWarps = EP_WARPS;            // warps per CTA: one per voxel-row pair
constexpr int kThreads = kWarps * 32;
constexpr int kTileY = kWarps - 1;          // output rows per CTA (warps 1..kWarps-1)
constexpr int kMinBlocks = EP_MIN_BLOCKS;   // occupancy hint for the stencil kernels
constexpr int kTileX = 30;                  // output voxels per row (lanes 1..30)
constexpr int kMaxStim = 8;
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned short kNonTissue = 0xBC00u;  // fp16 -1.0: record lane 3 of a non-tissue voxel

enum Mode { M_APPLY = 0, M_RHS = 1, M_PAR_MONO = 2, M_PAR_BI = 3, M_JAC = 4 };

// One CTA's work: voxel columns x in [30 bx, 30 bx + 30), rows
// y in [kTileY by, kTileY by + kTileY), output planes [k0, k1).
struct Seg {
    int bx, by, k0, k1;
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
    int nseg;             // work items (CTAs)
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
    Ctl *ctl;             // JAC (and PAR: non-finite flag)
};

__device__ __forceinline__ float h2f(unsigned short b) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ bool rec_tissue(const ushort4 &r) { return (r.w & 0x8000u) == 0; }

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

}  // namespace gbep
