/*
 * ep.h -- C ABI of the GB300 voxel electrophysiology step.
 *
 * One time step of the operator-split, matrix-free finite-volume
 * bidomain / monodomain model of cardiac tissue on a voxel grid
 * (T. Simpson, "Computational Tools for Cardiac Simulation", thesis,
 * arXiv 2302.12519):
 *
 *   1. Mitchell-Schaeffer reaction, explicit Euler
 *      (Eqs. ms1/ms2, Sec. "Algorithm Details / Electrophysiology / Reaction");
 *   2. anisotropic diffusion with the self-dual 27-point operator, fibre
 *      conductivity tensors (Eq. sigma1) and no-flux faces at the tissue mask
 *      (Sec. "Operators", Sec. "Matrix-Free Assembly", Sec. "Diffusion");
 *   3. bidomain only: the extracellular elliptic equation (Eq. bidomain1,
 *      second line) by damped Jacobi (Eq. dampjac1), FP64 residual norms,
 *      and the zero-mean reference potential per tissue component.
 *
 * All compute runs in CUDA kernels on one GPU; the host only orchestrates.
 *
 * Conventions for every call
 *  - Every function returns an ep_status; nothing throws across the ABI.
 *    On failure ep_last_error() returns a message for that handle.
 *  - Host buffers passed in are copied before the call returns; the library
 *    keeps no pointer to caller memory.
 *  - Device memory is owned by the handle.  It is allocated with
 *    ep_grid_desc.dev_alloc / dev_free when both are set (e.g. a framework's
 *    caching allocator), otherwise with cudaMalloc / cudaFree.
 *  - All work is issued on ep_grid_desc.cuda_stream (NULL = the legacy
 *    default stream).  Calls that return host data synchronise that stream.
 *  - A handle is not thread safe: use it from one host thread at a time.
 *  - Grid: nx * ny * nz voxels, linear index q = i + nx*(j + ny*k).
 *    Units: mm, ms, mS/mm.  The state v is dimensionless (0 rest, 1 peak);
 *    potentials read in mV use V_m = 100 v - 80 and V_e = 100 v_e.
 */
#ifndef EP_H
#define EP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EP_OK = 0,
    EP_EINVAL = 1,      /* bad argument, size or parameter value */
    EP_ENOMEM = 2,      /* device or host allocation failed */
    EP_ECUDA = 3,       /* a CUDA call failed (message has the CUDA error) */
    EP_ENOCONV = 4,     /* elliptic solve hit max_iter (or diverged); step completed with the last iterate */
    EP_ENONFINITE = 5,  /* a NaN / Inf appeared in the state */
    EP_ESTATE = 6,      /* call not valid in the handle's current state */
    EP_EBUSY = 7,       /* batch slot table full */
    EP_EREJECTED = 8,   /* batch admission refused: over the HBM budget */
    EP_ECANCELLED = 9   /* served request cancelled before it finished */
} ep_status;

enum { EP_MONO = 0, EP_BI = 1 };          /* ep_grid_desc.model */
enum { EP_FP32 = 0, EP_FP64 = 1 };        /* ep_grid_desc.precision: state and stencil arithmetic */

/* fields for ep_read (always returned as n doubles) */
enum {
    EP_VM_MV = 0,   /* transmembrane potential, mV */
    EP_W = 1,       /* gating variable */
    EP_VE_MV = 2,   /* extracellular potential (zero mean per component), mV */
    EP_TACT = 3,    /* activation time, ms; -1 where not yet activated */
    EP_V = 4,       /* dimensionless v */
    EP_VE = 5       /* dimensionless v_e */
};

typedef struct {
    int nx, ny, nz;                  /* voxels per axis, each >= 1 */
    double dx_mm;                    /* voxel edge, > 0 */
    int model;                       /* EP_MONO or EP_BI */
    int precision;                   /* EP_FP32 or EP_FP64 */
    void *cuda_stream;               /* cudaStream_t, may be NULL */
    void *(*dev_alloc)(size_t bytes, void *ctx);   /* optional device allocator */
    void (*dev_free)(void *ptr, void *ctx);        /* optional, paired with dev_alloc */
    void *alloc_ctx;                 /* passed to dev_alloc / dev_free */
} ep_grid_desc;

typedef struct {
    /* Mitchell-Schaeffer constants (Eqs. ms1/ms2): ms, ms, ms, ms, dimensionless */
    double tau_in, tau_out, tau_open, tau_close, v_gate;
    /* conductivities (Eq. sigma1), mS/mm: intracellular and extracellular,
     * longitudinal and transverse */
    double sig_iL, sig_iT, sig_eL, sig_eT;
    double lambda;        /* monodomain ratio (Eq. monodomain1) */
    double K;             /* chi_m * C_m, > 0 */
    double dt_ms;         /* time step, > 0 */
    double jacobi_omega;  /* damping of Eq. dampjac1 (the thesis requires damping but gives no value):
                             > 0: that value, < 2;
                             0: 1.8 / (8 sL / (sL + 2 sT)), the Fourier bound of a uniform tensor, for
                             the elliptic operator's sL = sig_iL + sig_eL, sT = sig_iT + sig_eT;
                             < 0: estimated at set-up (bidomain): min(1, 1.9 / lmax), lmax the
                             largest eigenvalue of D^-1 A from the Lanczos estimate scaled by 1.05
                             (or cheb_lmax when given).  The value in use: ep_get_info's omega. */
    double rel_tol;       /* stop when ||b - A x||_2 <= rel_tol ||b||_2 */
    int check_every;      /* residual check interval in sweeps, >= 1 (both solves) */
    int max_iter;         /* sweep cap per solve, >= 1 (both solves) */
    int diffusion;        /* EP_EXPLICIT: the parabolic part by explicit Euler (default);
                             EP_IMPLICIT: by implicit Euler, (I + a L_i) v+ = v* for the monodomain
                             (a = dt/K lambda/(1+lambda)) or v* - a L_i ve^n for the bidomain
                             (a = dt/K, ve of step n), solved by the undamped Jacobi step of
                             Eq. iejac1 from v* to rel_tol (Sec. "Implicit Euler", "Diffusion").
                             Implicit handles are stepped by ep_step only, not in a batch. */
    int solver;           /* elliptic solve: EP_SOLVER_JACOBI, the damped Jacobi of Eq. dampjac1 (default);
                             EP_SOLVER_CHEBYSHEV, Golub and Varga's Chebyshev semi-iteration on
                             the Jacobi step (no counterpart in the paper, whose future work names
                             faster solvers).  FP32 bidomain handles run both in correction form:
                             the iterate is x0 + e, e iterated on A e = b - A x0 from e = 0 and
                             folded into x0 each time a cycle has cut ||r|| by 1e3 (the Chebyshev
                             polynomial restarts there), which keeps the FP32 rounding of the full
                             iterate out of the iteration; the stop rule applies to the residual of
                             x0 + e, and v_e is its FP32 rounding.  It costs a third iterate buffer
                             (4 bytes a voxel; ep_footprint counts it).  FP64 handles run the plain
                             iterations;
                             EP_SOLVER_GAUSS_SEIDEL, Gauss-Seidel (SOR with omega = jacobi_omega when
                             0 < jacobi_omega < 2, else omega = 1) over the eight colour classes
                             (i, j, k mod 2): the deterministic form of the paper's in-place Jacobi,
                             whose races read already-updated neighbours (Sec. "Jacobi method");
                             a sweep is eight colour passes, in place, its residual the sum of each
                             colour's residuals as its pass forms them.  Not with a torso, not in
                             a batch.  Same stop rule, FP64 norms and cap (in sweeps). */
    double cheb_lmin, cheb_lmax;  /* EP_SOLVER_CHEBYSHEV: interval of the eigenvalues of D^-1 A that the
                             polynomial targets (A the elliptic operator, D its diagonal as stored);
                             both <= 0: estimated at set-up (Lanczos, 40 steps), read back with
                             ep_get_info; else 0 < lmin < lmax */
} ep_params;

#define EP_EXPLICIT 0
#define EP_IMPLICIT 1
#define EP_SOLVER_JACOBI 0
#define EP_SOLVER_CHEBYSHEV 1
#define EP_SOLVER_GAUSS_SEIDEL 2

typedef struct {
    int iters;               /* Jacobi sweeps of the last elliptic solve (0 for monodomain) */
    double rel_res;          /* last checked relative residual */
    int converged;           /* 1 if every solve in the call met rel_tol */
    long long total_iters;   /* sweeps summed over the steps of the call */
    long long step;          /* step counter after the call (t = step * dt) */
    long long ie_total_iters;   /* implicit-diffusion Jacobi sweeps summed over the steps of the call */
} ep_step_stats;

typedef struct {
    long long n_voxels;      /* nx * ny * nz */
    long long n_tissue;      /* tissue voxels */
    int n_components;        /* face-connected tissue components */
    int n_segments;          /* z-march work items of the stencil kernels */
    double omega;            /* damping in use */
    size_t device_bytes;     /* device memory held by the handle */
    double cheb_lmin, cheb_lmax;   /* interval of D^-1 A in use: the Chebyshev solver's, or the estimate behind
                                      an estimated jacobi_omega; 0 when neither needs one */
    long long n_domain;      /* voxels of the elliptic equation: tissue, plus the torso if set */
    int n_segments_elliptic; /* work items of the elliptic sweeps (n_segments without a torso) */
    int n_segments_far;      /* of those, items whose voxels and halo hold no tissue (swept by the
                                single-term kernel: there the operator is the torso's alone) */
} ep_info;

typedef struct ep_sim ep_sim;

/* Create a handle for one simulation.  Validates the descriptor (EP_EINVAL),
 * creates no device state until the first ep_step / ep_read / ep_apply_operator. */
ep_status ep_create(const ep_grid_desc *desc, ep_sim **out);

/* Tissue mask, n = nx*ny*nz bytes, non-zero = myocardium.  Required. */
ep_status ep_set_mask(ep_sim *s, const uint8_t *mask, size_t n);

/* Fibre field, 3n floats (fx, fy, fz) per voxel: unit length, or zero
 * (Sigma = sigma_T I, Sec. "Fibre Directions"), or longer than 1 for a
 * fast-conducting fibre (Sigma = sigma_T I + (sigma_L - sigma_T) f f^T,
 * Eq. sigma1, so |f|^2 = (g sigma_L - sigma_T) / (sigma_L - sigma_T) gives
 * the longitudinal conductivity g sigma_L; such voxels may need a smaller
 * jacobi_omega than the default).  Components finite and at most 4 in
 * magnitude (EP_EINVAL).  Stored as given (float32).  Optional (default
 * zero fibres). */
ep_status ep_set_fibres(ep_sim *s, const float *f, size_t n3);

/* Model parameters.  Required.  Values are validated (EP_EINVAL). */
ep_status ep_set_params(ep_sim *s, const ep_params *p);

/* Add a stimulus box [lo, hi) in voxel indices: J_stim = amp_per_ms is added to
 * dv/dt of tissue voxels in the box while t_start <= t_n < t_start + dur, with
 * t_n = n * dt evaluated in double precision.  At most 8 boxes. */
ep_status ep_add_stimulus(ep_sim *s, const int lo[3], const int hi[3],
                          double t_start_ms, double dur_ms, double amp_per_ms);

/* The ep_set_mask/fibres/params/stimulus calls are valid only before device
 * setup (first ep_step / ep_read / ep_apply_operator / ep_set_state); after
 * that they return EP_ESTATE. */

/* Overwrite the state: v, w, ve as n doubles each (any may be NULL to keep the
 * current field), step counter.  Values off the tissue are ignored.  The
 * default initial state is rest: v = 0, w = 1, ve = 0, step 0. */
ep_status ep_set_state(ep_sim *s, const double *v, const double *w, const double *ve,
                       size_t n, long long step);

/* Advance n_steps >= 0 time steps.  Returns EP_ENOCONV if an elliptic solve hit
 * max_iter (the step is completed with the last iterate), EP_ENONFINITE if a
 * NaN/Inf appeared.  stats may be NULL. */
ep_status ep_step(ep_sim *s, int n_steps, ep_step_stats *stats);

/* Copy one field to host: bytes must be n * sizeof(double). */
ep_status ep_read(ep_sim *s, int field, void *host, size_t bytes);

/* Snapshot / restore of the full dynamic state (v, w, ve, activation times,
 * step) in the handle's precision.  ep_state_bytes gives the blob size. */
ep_status ep_state_bytes(ep_sim *s, size_t *bytes);
ep_status ep_read_state(ep_sim *s, void *host, size_t bytes);
ep_status ep_write_state(ep_sim *s, const void *host, size_t bytes);

/* Apply the diffusion operator L_{sL,sT} = G'^T S G' of the handle's mask and
 * fibres to a host field u (n doubles), writing L u (n doubles; zero off the
 * tissue).  L u approximates -div(Sigma grad u) (Sec. "Operators / Laplacian",
 * Eq. ass3).  Uses the same stencil kernel as the time step. */
ep_status ep_apply_operator(ep_sim *s, double sig_L, double sig_T,
                            const double *u_host, double *out_host, size_t n);

ep_status ep_get_info(ep_sim *s, ep_info *info);

/* Conducting torso around the heart (Eq. bidomain1, lines 3-5; Sec.
 * "Electrocardiogram": the extracellular potential spreads into the
 * surrounding body, whose conductivity is a free parameter).  torso: n bytes,
 * non-zero = a torso voxel; voxels that are also tissue stay tissue.  sig_o:
 * the torso's isotropic conductivity (mS/mm, finite and > 0).  The elliptic
 * equation then acts on tissue + torso, with Sigma_i + Sigma_e on the tissue
 * and sig_o I on the torso under the same vertex averaging, so v_e and the
 * extracellular current are continuous across the heart surface and no
 * current leaves the outer surface of the torso; the right-hand side
 * -L_i v and the membrane state stay on the tissue, and the reference
 * potential is zero mean per face-connected component of tissue + torso.
 * Bidomain with explicit diffusion only (EP_EINVAL at set-up otherwise);
 * not for the batched or served forms.  An all-zero torso removes it.
 * Valid only before set-up (EP_ESTATE). */
ep_status ep_set_torso(ep_sim *s, const uint8_t *torso, size_t n, double sig_o);

/* ECG (Sec. "Electrocardiogram"): three electrode voxels (i, j, k) of the
 * right arm, left arm and left leg, in that order (9 ints), on tissue or
 * torso (checked at set-up, EP_EINVAL).  After every step's elliptic solve
 * the device records the three potentials; capacity is the number of samples
 * it holds between ep_read_ecg calls, and a step that would exceed it returns
 * EP_EBUSY without running.  capacity 0 switches the ECG off.  Bidomain only;
 * valid only before set-up (EP_ESTATE). */
ep_status ep_set_ecg(ep_sim *s, const int electrodes[9], int capacity);

typedef struct {
    double t_ms;             /* time at the end of the step */
    double phi_mV[3];        /* electrode potentials RA, LA, LL: 100 v_e */
    double lead_mV[6];       /* I = LA - RA, II = LL - RA, III = LL - LA, aVR = RA - (LA + LL)/2,
                                aVL = LA - (RA + LL)/2, aVF = LL - (RA + LA)/2 */
} ep_ecg_sample;

/* Moves the samples recorded since the last call into out (oldest first) and
 * empties the record; *n_out = their number.  max_samples below that number
 * gives EP_EINVAL with the number in *n_out and nothing moved.  Synchronises
 * the handle's stream. */
ep_status ep_read_ecg(ep_sim *s, ep_ecg_sample *out, int max_samples, int *n_out);

/* Apply the elliptic operator of the handle (L_i + L_e, plus the torso's
 * sig_o I if set) to a host field u (n doubles), writing n doubles (zero
 * outside tissue + torso), with the same kernel as the solve's sweeps.
 * Diagnostic. */
ep_status ep_apply_elliptic(ep_sim *s, const double *u_host, double *out_host, size_t n);

/* Same as ep_step, but the call allocates no device memory.  (The paper has
 * no counterpart; this serves embedding code.)  Some callers cannot allocate
 * while they advance the model: code that plans all device memory up front
 * (a framework that forbids library allocations after initialisation, a
 * real-time loop that must not block in the allocator, a multi-tenant
 * service with a fixed memory budget).  Here the step's scratch (the
 * elliptic solve's control block, its per-CTA FP64 partial sums, the
 * per-component means, and the non-finite flag) lives in one fixed device
 * array compiled into the library, about 290 KB, which every GPU that loads
 * the library holds until the process exits.  The rest of the state stays in
 * the handle: the handle must already be set up (one ep_step, ep_set_state
 * or ep_get_info call, which allocate), else EP_ESTATE.  Limits: at most
 * 32768 stencil work items (ep_info.n_segments) and 32768 reduction chunks
 * (2048 tissue voxels each), at most 4096 tissue components; larger problems
 * get EP_EINVAL with a message.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current,
 * and looks it up again when the device's context has changed since (after
 * a cudaDeviceReset the handle itself must be created anew: its device
 * memory went with the old context); make that first call before any stream
 * capture.  All calls on a device
 * share the one array and each call clears it first: calls whose work
 * overlaps on the GPU (several handles on concurrent streams) race on it,
 * so run them one after another.  Sweeps are launched one by one, without
 * the CUDA graph that ep_step uses. */
ep_status ep_step_noalloc(ep_sim *s, int n_steps, ep_step_stats *stats);

/* Device-time accounting of ep_step, measured with CUDA events on the
 * handle's stream (for throughput and roofline reporting).  Enabling resets
 * the counters; enabled accounting adds one event pair per kernel group. */
typedef struct {
    double sweep_ms;             /* Jacobi sweep launches (the elliptic solve) */
    double other_ms;             /* reaction+diffusion, right-hand side, reductions, projection */
    long long sweep_launches;    /* sweep kernels launched, including ones that found the solve finished */
    long long sweeps;            /* sweeps that did work */
    long long other_launches;    /* all other kernels launched by ep_step */
    long long steps;             /* steps taken while enabled */
    double ie_sweep_ms;          /* implicit-diffusion sweep launches (included in other_ms) */
    long long ie_sweeps;         /* implicit-diffusion sweeps that did work */
} ep_profile;

/* Device memory of the handle, from a host-side plan of its mask (face-
 * connected components, reduction chunks, work items) made without touching
 * the device: resident_bytes is what the handle holds once set up, peak_bytes
 * the most it holds during set-up (staging of fibres, mask and records).
 * After set-up both equal the bytes held.  EP_ESTATE without a mask,
 * EP_EINVAL if the mask has no tissue.  Host-only; needs no GPU.  No
 * counterpart in the paper: admission control of the served form. */
ep_status ep_footprint(ep_sim *s, size_t *resident_bytes, size_t *peak_bytes);

ep_status ep_profile_enable(ep_sim *s, int on);
ep_status ep_get_profile(ep_sim *s, ep_profile *prof);

/* ------------------------------------------------------------------------ */
/* Batched form: many instances advance together.                            */
/* ------------------------------------------------------------------------ */
/* The thesis proposes running many cardiac simulations in parallel on one
 * GPU; this is that form.  Uneven FP32 instances (different grids,
 * conductivities, stimuli) are advanced together.  Each kernel of a step is
 * one persistent launch over the packed list of all instances' work items.
 * Every instance keeps its own elliptic solve: its own sweep count, FP64
 * residual and stop flag.  A whole chunk of steps, including every
 * convergence loop, is one CUDA graph with device-side loop conditions, so
 * the host is not involved between steps.  Results per instance are the same
 * as ep_step on that instance alone, up to the order of the FP64 reductions
 * (which does not change either). */
typedef struct ep_batch ep_batch;

typedef struct {
    int instances;               /* instances in the batch */
    long long stencil_items;     /* packed stencil work items per launch */
    long long chunk_items;       /* packed reduction chunks per launch */
    size_t device_bytes;         /* device memory of the member handles */
    size_t budget_bytes;         /* admission budget */
    int sweeps_per_check;        /* sweep launches between device loop checks (set or tuned; untouched,
                                    each group takes about 1 ms of its sweeps, 8..64) */
    int zseg;                    /* z-planes per stencil work item (tuned) */
    size_t group_bytes;          /* members are swept in groups whose working sets total at most
                                    this many bytes, so a group's sweeps stay in L2 (0 = one group; tuned) */
    int groups;                  /* number of such groups */
    int solo_members;            /* members whose Jacobi sweeps run as their own launches, concurrent
                                    with the packed launch of the others: those with at least half a
                                    wave of stencil items (3 CTAs per SM x SMs / 2, 228 on 152 SMs),
                                    and every member of a group of at most 8 */
} ep_batch_info;

/* Create a batch of at most max_instances handles whose device memory may
 * total at most hbm_budget_bytes (0 = no budget).  cuda_stream may be NULL. */
ep_status ep_batch_create(int max_instances, size_t hbm_budget_bytes, void *cuda_stream, ep_batch **out);

/* Admit a handle (FP32, same model as the batch's other members; it is set up
 * here if needed).  The batch does not own it: the caller keeps it alive until
 * ep_batch_remove and reads results with ep_read on it.  EP_EREJECTED if its
 * device memory would exceed the budget, EP_EBUSY if the batch is full.
 * *slot receives the slot number. */
ep_status ep_batch_add(ep_batch *b, ep_sim *sim, int *slot);
ep_status ep_batch_remove(ep_batch *b, int slot);

/* Advance every member n_steps time steps (one graph launch). */
ep_status ep_batch_step(ep_batch *b, int n_steps);

/* Per-member statistics of the last ep_batch_step (iters of its last solve,
 * whether every solve converged, its step counter). */
ep_status ep_batch_slot_stats(ep_batch *b, int slot, ep_step_stats *stats);

/* Choose the z-planes per work item and the group size by timing
 * trial_sweeps sweeps of each candidate on the members' current states
 * (states are restored afterwards); the sweeps per device loop check follow
 * from the measured sweep time (about 1 ms of sweeps, 8..64). */
ep_status ep_batch_autotune(ep_batch *b, int trial_sweeps);

/* Set the schedule by hand: sweep launches between device loop checks
 * (1..1024), z-planes per work item (8..256) and the group budget in bytes.
 * 0 (or a negative group_bytes) keeps a value.  Results do not depend on the
 * schedule. */
ep_status ep_batch_set_schedule(ep_batch *b, int sweeps_per_check, int zseg, long long group_bytes);

ep_status ep_batch_get_info(ep_batch *b, ep_batch_info *info);
const char *ep_batch_last_error(const ep_batch *b);
void ep_batch_destroy(ep_batch *b);

/* ------------------------------------------------------------------------ */
/* Served form: a request loop with continuous batching.                     */
/* ------------------------------------------------------------------------ */
/* The paper suggests running many cardiac simulations side by side rather
 * than splitting one across processors (chapter "Review & Outlook", Sec.
 * "Assesment"); it has no serving loop, so nothing here has a counterpart in
 * it.
 *
 * A server owns a serving thread and one batch per model.  A request is a
 * prepared FP32 handle (mask and parameters set; fibres and stimuli
 * optional) plus a step count and a release time.  Released requests are
 * admitted in release order while a slot is free and the request's set-up
 * peak (ep_footprint) fits the budget next to the bytes of every request the
 * server holds (running or finished and not yet collected); a request whose
 * peak alone exceeds the budget finishes with EP_EREJECTED.  Admitted
 * requests are set up on the device and stepped with the other members in
 * chunks of at most chunk_steps steps; a chunk never takes a member past its
 * step count, and requests join or leave only between chunks.  Each request
 * computes exactly what ep_step on the handle alone computes.
 *
 * Ownership: ep_server_submit hands the handle to the server; it comes back
 * in the ep_request_result of ep_server_collect (state on the device, read
 * with ep_read; the caller destroys it).  ep_server_destroy destroys the
 * handles it still holds.  All functions may be called from any host thread. */
typedef struct ep_server ep_server;

typedef struct {
    int max_slots;              /* requests stepped together, >= 1 */
    int chunk_steps;            /* steps between admission points, >= 1 */
    int sweeps_per_check;       /* batch schedule (ep_batch_set_schedule); 0 = default */
    size_t hbm_budget_bytes;    /* device bytes the held requests may total; 0 = no limit */
    void *cuda_stream;          /* stream of the batched launches; NULL = a private one */
    long long max_active_items; /* admit while the running requests' stencil work items (one z-march
                                   tile each) stay within this many; a request is always admitted onto an
                                   idle device; 0 = no limit */
} ep_server_config;

typedef struct {
    long long id;
    int status;                 /* EP_OK, EP_ENOCONV (some solve hit max_iter; all steps done),
                                   EP_ENONFINITE, EP_ECANCELLED, EP_EREJECTED, or the set-up error */
    int steps_done;
    long long n_tissue;
    long long total_iters;      /* Jacobi sweeps of the request's solves */
    double t_release_s, t_admit_s, t_done_s;   /* server clock (ep_server_now); t_admit_s < 0: never admitted */
    size_t device_bytes;        /* device memory the handle holds */
    ep_sim *sim;                /* the handle, returned to the caller */
} ep_request_result;

typedef struct {
    int queued, active, finished;   /* finished = retired and not collected */
    long long submitted, admitted, completed, cancelled, rejected;
    long long chunks;               /* batched chunks run */
    long long voxel_steps;          /* tissue voxel-steps done */
    size_t hbm_in_use, hbm_peak;    /* bytes held (set-up reservations included), and the maximum */
    double busy_s;                  /* wall time spent in batched chunks */
    double now_s;
} ep_server_stats;

/* Start a server on the current device.  EP_ECUDA without a usable device. */
ep_status ep_server_create(const ep_server_config *cfg, ep_server **out);

/* Queue a request that is released at release_s on the server clock (a time
 * already past means now).  *id receives its id.  EP_EINVAL for FP64 handles
 * or a handle the server already holds. */
ep_status ep_server_submit(ep_server *srv, ep_sim *sim, int n_steps, double release_s, long long *id);

/* Cancel a queued request at once, or a running one at the next chunk
 * boundary (status EP_ECANCELLED, steps_done says how far it got). */
ep_status ep_server_cancel(ep_server *srv, long long id);

/* Take up to max_results finished requests, waiting up to wait_s seconds for
 * the first one.  *n_out = number returned (0 after a timeout). */
ep_status ep_server_collect(ep_server *srv, ep_request_result *out, int max_results, int *n_out, double wait_s);

/* Wait until no request is queued or running (timeout_s < 0: no limit);
 * EP_EBUSY at the timeout.  Finished requests keep their device memory until
 * collected, so under a tight budget admission can wait on the caller:
 * drain then returns EP_EBUSY at once (nothing runs, the next request needs
 * memory that uncollected results hold).  Collect and drain again. */
ep_status ep_server_drain(ep_server *srv, double timeout_s);

ep_status ep_server_get_stats(ep_server *srv, ep_server_stats *out);
double ep_server_now(const ep_server *srv);
const char *ep_server_last_error(const ep_server *srv);
void ep_server_destroy(ep_server *srv);
const char *ep_last_error(const ep_sim *s);
void ep_destroy(ep_sim *s);

#ifdef __cplusplus
}
#endif
#endif /* EP_H */
