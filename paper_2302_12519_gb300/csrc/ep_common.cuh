// ep_common.cuh -- shared definitions of the sm_103a kernels of the voxel
// electrophysiology step: work items, the per-instance descriptor and control
// block, the Mitchell-Schaeffer update and a fixed-order block reduction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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
constexpr float kNonTissueW = -1.0f;           // record lane 3 of a voxel outside the records' domain
constexpr unsigned kBathTag = 0x80000000u;      // -0.0f in lane 0: a torso voxel of the elliptic records
constexpr int kRedThreads = 256;            // reduction kernels
constexpr int kChunk = 2048;                // tissue voxels per reduction chunk

// M_IE_RHS: reaction plus f = v* - a L_i ve of the implicit bidomain step;
// M_IE: one Jacobi sweep of (I + a L_i) x = f (Eq. iejac1);
// M_JAC_BATH, M_APPLY_BATH: the elliptic sweep and operator over tissue + a
// conducting torso (Eq. bidomain1, lines 3-5): the tissue term (pairs of
// tissue voxels, fibre tensors) plus the torso term (pairs of any two domain
// voxels, sig_o I per torso voxel of the vertex block).
// M_JAC_CHEB, M_JAC_BATH_CHEB: the same sweeps accelerated by the Chebyshev
// semi-iteration (separate instances, so the plain sweeps carry none of it).
// M_JAC_GS: one colour pass of the eight-colour Gauss-Seidel / SOR sweep, in
// place on x0 (a sweep is eight launches, colours 0..7).
enum Mode { M_APPLY = 0, M_RHS = 1, M_PAR_MONO = 2, M_PAR_BI = 3, M_JAC = 4, M_IE_RHS = 5, M_IE = 6, M_JAC_BATH = 7,
            M_APPLY_BATH = 8, M_JAC_CHEB = 9, M_JAC_BATH_CHEB = 10, M_JAC_GS = 11 };
enum Diffusion { DIFF_EXPLICIT = 0, DIFF_IMPLICIT = 1 };

// Modes that run a solve sweep (Jacobi of the elliptic or the implicit parabolic system).
template <int MODE>
constexpr bool kCheb = MODE == M_JAC_CHEB || MODE == M_JAC_BATH_CHEB;
template <int MODE>
constexpr bool kGS = MODE == M_JAC_GS;
template <int MODE>
constexpr bool kJac = MODE == M_JAC || MODE == M_JAC_BATH || kCheb<MODE> || kGS<MODE>;
template <int MODE>
constexpr bool kTwoTerm = MODE == M_JAC_BATH || MODE == M_APPLY_BATH || MODE == M_JAC_BATH_CHEB;
template <int MODE>
constexpr bool kSweep = kJac<MODE> || MODE == M_IE;
enum Model { MODEL_MONO = 0, MODEL_BI = 1 };

// One stencil work item: voxel columns x in [x0, x0 + 30), rows
// y in [kTileY by, kTileY by + kTileY), output planes [k0, k1).
struct Seg {
    int x0, by, k0, k1;
};

struct StimBox {
    int lo[3], hi[3];
    double t0, t1;        // active while t0 <= t_n < t1 (t1 = t_start + dur, formed in double)
    double amp;
};

struct StimSet {
    int n;
    StimBox box[kMaxStim];
};

// Device control block of one instance: step counter and the elliptic solve.
struct Ctl {
    unsigned int arrive;  // work items that finished the current launch (reset by the last one)
    int done;             // solve finished: converged, capped, diverged or empty rhs
    int sweep;            // sweeps done in the current solve, as of its last residual check
    int iters;            // sweeps of the finished solve
    int converged;
    int nonfinite;
    int diverged;
    int noconv;           // some solve of this run hit max_iter or diverged
    double bnorm2;        // ||b||^2 after the mean correction
    double thresh2;       // rel_tol^2 * ||b||^2
    double rnorm2;        // ||r||^2 at the last check
    long long step;       // time step n (t_n = n dt); v, w of step n live in buffer n & 1
    long long total_iters;
    // work items of the current solve that finished a sweep, cumulative: when an item of sweep j
    // starts, every item of sweeps < j has arrived and fewer than nitems of sweep j have, so
    // jarrive / nitems = j; sweeps that do not check the residual only add to it
    unsigned long long jarrive;
    long long ie_total;   // sweeps of the implicit parabolic solves, summed over steps
    // Chebyshev solve in correction form: the sweep that starts the current cycle, and
    // ||r||^2 at that cycle's start
    int cycle0, pad_c;
    double r0n2;
};

struct Chunk {
    int start, end, comp;  // [start, end) into the component-sorted tissue index list
};

// Everything a kernel needs about one simulation instance.  Passed by value
// to the single-instance kernels and read from a device table by the
// batched ones.
template <typename real>
struct Inst {
    int nx, ny, nz, model;
    int nseg, nchunk, ncomp, check_every;
    int max_iter, pad;
    const Seg *segs;
    const float4 *rec;    // (fx, fy, fz, 1/Dhat) in fp32; lane 3 = -1 off the records' domain
    real *v[2], *w[2];    // state, buffer = step & 1
    real *x0, *x1;        // elliptic iterates; x0 holds v_e between steps
    real *b;              // elliptic right-hand side
    real *tact;           // activation times
    const int *idx;       // component-sorted tissue voxels
    const Chunk *chunks;
    const int *comp_chunk0;
    const long long *comp_count;
    double *means, *partials;
    Ctl *ctl;
    real sTi, dSi;        // intracellular operator: sigma_T, sigma_L - sigma_T
    real sTie, dSie;      // elliptic operator (intra + extra)
    real C;               // 1 / (8 dx^2)
    real coef_par;        // dt / K (times lambda / (1 + lambda) for the monodomain)
    real coef_jac;        // omega / C
    real dt, inv_tin, inv_tout, inv_topen, inv_tclose, vgate;
    double dt_d, rel_tol2, div_factor;
    StimSet stim;
    // implicit-Euler diffusion (diffusion == DIFF_IMPLICIT): second iterate buffer,
    // 1 / (1 + a D_i) per voxel and a = dt/K (times lambda/(1+lambda) for the monodomain)
    int diffusion, pad2;
    real *ie_x;
    const real *ie_inv;
    real alpha_ie;
    // Chebyshev semi-iteration of the elliptic solve (solver == 1): tau / C for the
    // basic step, rho and theta = acosh(1 / rho) for the weights; solver == 2 is the
    // eight-colour Gauss-Seidel / SOR solve (coef_jac = omega / C)
    int solver, pad3;
    real cheb_tau_c;
    double cheb_rho, cheb_theta;
    // conducting torso: the elliptic descriptor's records tag torso voxels (kBathTag), and
    // sig_o is the torso term's conductivity; in the tissue descriptor the reductions of the
    // elliptic right-hand side count torso voxels as 0
    int torso, pad4;
    real sig_o;
    // a sweep split over two launches (torso handles: items far from the tissue run the
    // single-term kernel): this launch's first item among the sweep's items, and their count
    // (0: the launch is the whole sweep)
    int item0, nitems_all;
    // elliptic solve in correction form (FP32 handles, damped Jacobi and Chebyshev): the iterate
    // is x0 + e, e in x1 / x2 (sweep j >= 1 reads e_j from x1 when j is odd, else from x2), b holds
    // the residual of x0 at the cycle's start; a cycle restarts from e = 0 once it has cut ||r||
    // by a factor 1e3 (kRestart2)
    real *x2;
    int eform, pad5;
};

// A correction-form cycle restarts when ||r||^2 has fallen below this fraction of
// its value at the cycle's start (a factor 1e3 in the norm).
constexpr double kRestart2 = 1e-6;

// Weight of sweep k of the Chebyshev semi-iteration: w = 1 for k = 0, else
// w_{k+1} = 2 T_k(1/rho) / (rho T_{k+1}(1/rho)) in the overflow-free form
// (2 / rho) e^-theta (1 + e^-2k theta) / (1 + e^-2(k+1) theta).
__device__ __forceinline__ double cheb_weight(int k, double rho, double theta)
{
    if (k == 0) return 1.0;
    const double a = exp(-2.0 * theta * k);
    return (2.0 / rho) * exp(-theta) * (1.0 + a) / (1.0 + a * exp(-2.0 * theta));
}

// A record is in its domain (tissue, or tissue + torso) when the sign bit of lane 3 is clear.
__device__ __forceinline__ bool rec_tissue(const float4 &r) { return __float_as_int(r.w) >= 0; }
__device__ __forceinline__ bool rec_bath(const float4 &r) { return __float_as_uint(r.x) == kBathTag; }

// Mitchell-Schaeffer explicit Euler (Eqs. ms1, ms2; closing branch -w/tau_close).
template <typename real>
__device__ __forceinline__ void ms_step(const Inst<real> &I, double tn, real v, real w, int x, int y, int z,
                                        real &vstar, real &wnew)
{
    real js = 0;
    for (int s = 0; s < I.stim.n; ++s) {
        const StimBox &bx = I.stim.box[s];
        if (tn >= bx.t0 && tn < bx.t1 && x >= bx.lo[0] && x < bx.hi[0] && y >= bx.lo[1] && y < bx.hi[1] &&
            z >= bx.lo[2] && z < bx.hi[2])
            js += real(bx.amp);
    }
    real jin = v * v * (real(1) - v) * w * I.inv_tin;
    real jout = -v * I.inv_tout;
    vstar = v + I.dt * (jin + jout + js);
    real dw = (v < I.vgate) ? (real(1) - w) * I.inv_topen : -w * I.inv_tclose;
    wnew = w + I.dt * dw;
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

// Arrival of one work item of an instance; true in the CTA that completes the
// launch for that instance (all its items' partial results are visible).
__device__ __forceinline__ bool arrive_last(Ctl *ctl, int nitems, int *sflag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *sflag = (atomicAdd(&ctl->arrive, 1u) == (unsigned)nitems - 1u);
    }
    __syncthreads();
    const bool last = *sflag != 0;
    if (last) __threadfence();
    return last;
}

// Entry of the list of unfinished members of a batched solve: prefix count of
// the items before it, its descriptor row and its control block.
struct ActRec {
    int cum, inst;
    Ctl *ctl;
};

// Work item of a batched launch: instance, item index within the instance,
// and the instance's item count.
struct BItem {
    int inst, item, nitems, pad;
};

}  // namespace gbep
