// ep_api.cu -- C ABI of the GB300 voxel electrophysiology step (see include/ep.h).
//
// Host side: validation, set-up of the data layout (fp32 fibre records,
// z-march segment list, component-sorted tissue index list), and the step
// orchestration.  Every arithmetic step of the time step runs in the kernels
// of ep_kernels.cuh.
//
// Elliptic solve control: the sweep count, residual checks and the stop
// decision live in a device control block.  Sweeps are queued in CUDA-graph
// chunks; a sweep that finds the solve finished returns at once, so the host
// only needs to look at the flag once per chunk (one chunk of look-ahead) and
// never stalls the GPU between sweeps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <cuda.h>

#include "../../include/ep.h"
#include "ep_kernels.cuh"

using namespace gbep;

namespace {

#ifndef EP_ZSEG
#define EP_ZSEG 16
#endif
constexpr int kZSeg = EP_ZSEG;     // default output planes per z-march segment
constexpr int kZSegMin = 8;        // smallest segment length the batch autotuner tries
constexpr int kSweepChunk = 64;    // sweeps per queued graph chunk
constexpr int kSoloAllMembers = 8; // batch groups this small sweep every member in its own launches
constexpr double kDivFactor = 1e16;

struct StimDef {
    int lo[3], hi[3];
    double t0, dur, amp;
};

}  // namespace

// Host-side layout of a handle, computed from the mask alone (before any
// device memory exists): the voxels of the elliptic domain (the tissue, plus
// the torso if one is set) sorted by face-connected component, reduction
// chunks, and the z-march work items of the tissue and of the domain.
struct HostPlan {
    bool done = false;
    std::vector<int> order;             // domain voxels, sorted by component then index
    std::vector<long long> comp_count;  // voxels per component
    std::vector<Chunk> chunks;
    std::vector<int> comp_chunk0;       // first chunk of each component (+ end)
    std::vector<Seg> segs;              // work items at the handle's z-planes per item
    std::vector<Seg> segs_z[4];         // work items at kZLens[i] planes per item (set-up picks one)
    std::vector<Seg> segs_e, segs_e_z[4];   // the same over the domain (torso handles only)
};

constexpr int kZLens[4] = {8, 16, 24, 32};

struct ep_sim {
    ep_grid_desc d{};
    long long n = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<uint8_t> mask;
    std::vector<float> fib;
    bool have_mask = false, have_params = false;
    ep_params p{};
    std::vector<StimDef> stims;
    std::vector<uint8_t> torso;  // conducting torso voxels outside the tissue (empty: none)
    double sig_o = 0.0;          // its conductivity (mS/mm)
    int ecg_q[3] = {-1, -1, -1}; // electrode voxels RA, LA, LL (-1: no ECG)
    long long ecg_cap = 0;       // samples the device record holds between reads
    HostPlan plan;
    size_t fp_resident = 0, fp_peak = 0;   // device bytes after / during set-up (from the plan)
    bool ready = false;
    // derived layout
    long long n_tissue = 0;
    long long n_domain = 0;      // voxels of the elliptic equation (tissue + torso)
    int ncomp = 0, nseg = 0, nchunk = 0;
    int nseg_e = 0;              // work items of the elliptic sweeps (nseg without a torso)
    int nseg_far = 0;            // the first of them, whose cells and halo hold no tissue
    int zseg = kZSeg;            // z-planes per stencil work item
    long long max_items = 0;     // segment capacity of the segs / partials buffers
    double omega = 0.0;
    double cheb_lmin = 0.0, cheb_lmax = 0.0;   // Chebyshev interval in use
    size_t rsz = 4;
    // device memory
    std::vector<void *> allocs;
    size_t dev_bytes = 0;
    float4 *rec = nullptr;
    float4 *rec_e = nullptr;    // records of the elliptic domain (rec without a torso)
    Seg *segs_e = nullptr;       // work items of the elliptic sweeps (segs without a torso)
    double *ecg = nullptr;       // ECG record: 3 potentials per sample
    long long ecg_n = 0;         // samples recorded since the last read
    double ecg_t0 = 0.0;         // time of the first of them (ms)
    void *v[2] = {nullptr, nullptr}, *w[2] = {nullptr, nullptr}, *x[2] = {nullptr, nullptr};
    void *b = nullptr, *tact = nullptr;
    Seg *segs = nullptr;
    int *idx = nullptr;
    Chunk *chunks = nullptr;
    int *comp_chunk0 = nullptr;
    long long *comp_count = nullptr;
    double *means = nullptr, *partials = nullptr;
    Ctl *ctl = nullptr;
    Ctl *ctl_host = nullptr;   // pinned, 2 slots
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaGraphExec_t sweep_graph = nullptr;
    cudaGraphExec_t ie_graph = nullptr;   // implicit-diffusion sweeps
    void *ie_x = nullptr, *ie_inv = nullptr;
    void *x2 = nullptr;          // second correction buffer of the FP32 elliptic solve (correction form)
    long long ie_seen = 0;                // implicit sweeps counted by earlier calls
    long long step = 0;
    bool noalloc_call = false;   // inside ep_step_noalloc: scratch is the static array, no graph
    // device-time accounting (ep_profile_enable)
    bool prof_on = false;
    cudaEvent_t pev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    ep_profile prof{};
};

namespace {

ep_status fail(ep_sim *s, ep_status st, const std::string &msg)
{
    if (s) s->err = msg;
    return st;
}

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(s, EP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)

void *dalloc(ep_sim *s, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (s->d.dev_alloc && s->d.dev_free) {
        p = s->d.dev_alloc(bytes, s->d.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        s->allocs.push_back(p);
        s->dev_bytes += bytes;
    }
    return p;
}

void dfree_all(ep_sim *s)
{
    for (void *p : s->allocs) {
        if (s->d.dev_alloc && s->d.dev_free) s->d.dev_free(p, s->d.alloc_ctx);
        else cudaFree(p);
    }
    s->allocs.clear();
    s->dev_bytes = 0;
}

// CTAs of a stencil launch: one per work item (segment)
int stencil_blocks(const ep_sim *s) { return std::max(1, s->nseg); }

int grid_for(long long n, int threads)
{
    long long g = (n + threads - 1) / threads;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

bool params_ok(const ep_params &p, std::string &why)
{
    auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    if (!pos(p.tau_in) || !pos(p.tau_out) || !pos(p.tau_open) || !pos(p.tau_close)) { why = "time constants must be > 0"; return false; }
    if (!std::isfinite(p.v_gate)) { why = "v_gate must be finite"; return false; }
    if (!pos(p.sig_iL) || !pos(p.sig_iT) || !pos(p.sig_eL) || !pos(p.sig_eT)) { why = "conductivities must be > 0"; return false; }
    if (!std::isfinite(p.lambda) || p.lambda <= 0.0) { why = "lambda must be > 0"; return false; }
    if (!pos(p.K) || !pos(p.dt_ms)) { why = "K and dt_ms must be > 0"; return false; }
    if (!std::isfinite(p.jacobi_omega) || p.jacobi_omega >= 2.0) { why = "jacobi_omega must be < 2 (0: the bound rule, < 0: estimated)"; return false; }
    if (!std::isfinite(p.rel_tol) || p.rel_tol < 0.0) { why = "rel_tol must be >= 0"; return false; }
    if (p.check_every < 1 || p.max_iter < 1) { why = "check_every and max_iter must be >= 1"; return false; }
    if (p.diffusion != EP_EXPLICIT && p.diffusion != EP_IMPLICIT) { why = "diffusion must be EP_EXPLICIT or EP_IMPLICIT"; return false; }
    if (p.solver != EP_SOLVER_JACOBI && p.solver != EP_SOLVER_CHEBYSHEV && p.solver != EP_SOLVER_GAUSS_SEIDEL) {
        why = "solver must be EP_SOLVER_JACOBI, EP_SOLVER_CHEBYSHEV or EP_SOLVER_GAUSS_SEIDEL";
        return false;
    }
    if (p.solver == EP_SOLVER_CHEBYSHEV && !(p.cheb_lmin <= 0.0 && p.cheb_lmax <= 0.0) &&
        !(std::isfinite(p.cheb_lmin) && std::isfinite(p.cheb_lmax) && p.cheb_lmin > 0.0 && p.cheb_lmin < p.cheb_lmax)) {
        why = "Chebyshev interval must satisfy 0 < cheb_lmin < cheb_lmax (both <= 0: estimated)";
        return false;
    }
    return true;
}

// Stencil work items.  The grid is cut into bands of kTileY rows and blocks of
// zseg planes; within each (band, block) the x positions holding tissue are
// covered greedily by windows of kTileX columns, each starting at the first
// tissue column not yet covered, and each window's planes are trimmed to the
// ones holding tissue.  The items partition the tissue voxels.  Placing the
// windows on the tissue, rather than on a fixed 30-column lattice, spends
// about 12 % fewer thread slots on the shell geometries.
// Torso handles: moves the work items whose voxels and one-voxel halo hold no
// tissue (the reach of their stencil) to the front, keeping the order within
// each class; returns their number.  There the elliptic operator is the torso
// term alone, which the single-term kernel computes with sigma = sig_o I.
int partition_far(std::vector<Seg> &segs, const uint8_t *heart, int nx, int ny, int nz)
{
    auto far = [&](const Seg &g) {
        const int xa = std::max(0, g.x0 - 1), xb = std::min(nx, g.x0 + kTileX + 1);
        const int ya = std::max(0, g.by * kTileY - 1), yb = std::min(ny, g.by * kTileY + kTileY + 1);
        const int za = std::max(0, g.k0 - 1), zb = std::min(nz, g.k1 + 1);
        for (int k = za; k < zb; ++k)
            for (int j = ya; j < yb; ++j) {
                const uint8_t *row = heart + (long long)nx * (j + (long long)ny * k);
                for (int i = xa; i < xb; ++i)
                    if (row[i]) return false;
            }
        return true;
    };
    auto mid = std::stable_partition(segs.begin(), segs.end(), far);
    return (int)(mid - segs.begin());
}

std::vector<Seg> build_segments(const uint8_t *m, int nx, int ny, int nz, int zseg)
{
    std::vector<Seg> segs;
    const int nby = (ny + kTileY - 1) / kTileY;
    std::vector<char> has((size_t)nz * nx);   // (plane, column) holds tissue in some row of the band
    std::vector<char> col(nx);
    for (int by = 0; by < nby; ++by) {
        const int ya = by * kTileY, yb = std::min(ya + kTileY, ny);
        for (int k = 0; k < nz; ++k) {
            char *h = &has[(size_t)k * nx];
            std::fill(h, h + nx, 0);
            for (int j = ya; j < yb; ++j) {
                const uint8_t *row = m + (long long)nx * (j + (long long)ny * k);
                for (int i = 0; i < nx; ++i) h[i] |= (char)(row[i] != 0);
            }
        }
        for (int kb = 0; kb < nz; kb += zseg) {
            const int ke = std::min(kb + zseg, nz);
            std::fill(col.begin(), col.end(), 0);
            for (int k = kb; k < ke; ++k)
                for (int i = 0; i < nx; ++i) col[i] |= has[(size_t)k * nx + i];
            for (int x0 = 0; x0 < nx; ++x0) {
                if (!col[x0]) continue;
                const int xe = std::min(x0 + kTileX, nx);
                int k0 = ke, k1 = kb;
                for (int k = kb; k < ke; ++k)
                    for (int i = x0; i < xe; ++i)
                        if (has[(size_t)k * nx + i]) {
                            k0 = std::min(k0, k);
                            k1 = std::max(k1, k + 1);
                            break;
                        }
                segs.push_back(Seg{x0, by, k0, k1});
                x0 = xe - 1;   // the next window starts past this one
            }
        }
    }
    // neighbouring tiles of one z-block run together (their shared halos hit L2)
    std::stable_sort(segs.begin(), segs.end(), [zseg](const Seg &a, const Seg &b) {
        if (a.k0 / zseg != b.k0 / zseg) return a.k0 / zseg < b.k0 / zseg;
        if (a.x0 != b.x0) return a.x0 < b.x0;
        return a.by < b.by;
    });
    return segs;
}

// ---------------------------------------------------------------------------
// set-up: layout built on the host from the mask, records on the device
// ---------------------------------------------------------------------------
size_t abytes(size_t b) { return b ? b : 16; }   // dalloc's size of a request

// Device bytes of a handle after set-up (resident) and during it (peak, which
// adds the staging buffers of fibres, mask and raw records).  Matches the
// allocations of setup_typed exactly.
#ifndef EP_LANCZOS_STEPS
#define EP_LANCZOS_STEPS 40
#endif
constexpr int kLanczosSteps = EP_LANCZOS_STEPS;
constexpr int kLanczosScalars = 2 + 2 * kLanczosSteps;   // alpha, beta of the current step; alpha_j, beta_{j+1}

// The set-up estimates the spectrum of D^-1 A for the Chebyshev solver and for the
// damped Jacobi's estimated damping.
bool needs_spectrum(const ep_sim *s)
{
    return s->p.solver == EP_SOLVER_CHEBYSHEV || (s->p.solver == EP_SOLVER_JACOBI && s->p.jacobi_omega < 0.0);
}

// Residual partial sums per stencil work item: one, or one per colour pass of the
// eight-colour sweep.
long long partial_slots(const ep_sim *s)
{
    const long long per = s->have_params && s->p.solver == EP_SOLVER_GAUSS_SEIDEL ? 8 : 1;
    return std::max<long long>(per * s->max_items, s->nchunk);
}

// Set-up scratch of the Chebyshev interval estimate (0 when the interval is
// given or the solver is damped Jacobi): the Lanczos scalars and two partial
// sums per reduction chunk.
size_t lanczos_bytes(const ep_sim *s)
{
    if (!s->have_params || s->d.model != EP_BI || s->p.cheb_lmin > 0.0) return 0;
    if (!needs_spectrum(s)) return 0;
    return sizeof(double) * ((size_t)kLanczosScalars + 2 * (size_t)s->nchunk);
}

// FP32 bidomain handles run the damped-Jacobi and Chebyshev solves in correction
// form (the FP32 rounding of the full iterate would floor the residual), which
// needs a third iterate buffer.
bool solve_eform(const ep_sim *s, size_t rb)
{
    return rb == sizeof(float) && s->have_params && s->d.model == EP_BI && s->p.solver != EP_SOLVER_GAUSS_SEIDEL;
}

void footprint(const ep_sim *s, size_t rb, size_t *resident, size_t *peak)
{
    const HostPlan &P = s->plan;
    const size_t n = (size_t)s->n;
    size_t r = abytes(sizeof(float4) * n) + 8 * abytes(rb * n);
    r += abytes(sizeof(Seg) * (size_t)s->max_items) + abytes(sizeof(int) * P.order.size());
    r += abytes(sizeof(Chunk) * P.chunks.size()) + abytes(sizeof(int) * P.comp_chunk0.size());
    r += abytes(sizeof(long long) * P.comp_count.size()) + abytes(sizeof(double) * (size_t)s->ncomp);
    r += abytes(sizeof(double) * (size_t)partial_slots(s)) + abytes(sizeof(Ctl));
    if (s->have_params && s->p.diffusion == EP_IMPLICIT) r += 2 * abytes(rb * n);   // second iterate, 1/(1 + a D)
    if (solve_eform(s, rb)) r += abytes(rb * n);
    const bool torso = !s->torso.empty();
    if (torso) r += abytes(sizeof(float4) * n) + abytes(sizeof(Seg) * (size_t)s->max_items);   // domain records, items
    if (s->ecg_q[0] >= 0) r += abytes(sizeof(double) * 3 * (size_t)s->ecg_cap);
    *resident = r;
    *peak = r + abytes(sizeof(float) * 3 * n) + abytes(n) + abytes(sizeof(float4) * n) + lanczos_bytes(s) +
            (torso ? abytes(n) : 0);
}

// Host analysis of the mask: face-connected components (breadth-first), the
// component-sorted tissue index list, reduction chunks and z-march segments.
// Fills s->plan and the derived counts; touches no device state.
ep_status plan_layout(ep_sim *s)
{
    if (s->plan.done) {   // the parameters may have changed since (implicit diffusion adds buffers)
        footprint(s, s->d.precision == EP_FP64 ? sizeof(double) : sizeof(float), &s->fp_resident, &s->fp_peak);
        return EP_OK;
    }
    if (!s->have_mask) return fail(s, EP_ESTATE, "ep_set_mask must be called first");
    const int nx = s->d.nx, ny = s->d.ny, nz = s->d.nz;
    const long long n = s->n;
    const bool torso = !s->torso.empty();
    std::vector<uint8_t> dom;   // elliptic domain: tissue or torso
    if (torso) {
        dom.resize(n);
        for (long long q = 0; q < n; ++q) dom[q] = (s->mask[q] || s->torso[q]) ? 1 : 0;
    }
    const uint8_t *m = torso ? dom.data() : s->mask.data();
    HostPlan &P = s->plan;
    std::vector<int> comp(n, -1);
    P.order.clear();
    P.order.reserve((size_t)std::count_if(s->mask.begin(), s->mask.end(), [](uint8_t c) { return c != 0; }));
    P.comp_count.clear();
    std::vector<long long> queue;
    int nc = 0;
    for (long long q = 0; q < n; ++q) {
        if (!m[q] || comp[q] >= 0) continue;
        queue.clear();
        queue.push_back(q);
        comp[q] = nc;
        size_t head = 0;
        while (head < queue.size()) {
            const long long c = queue[head++];
            const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
            const int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k}, {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
            for (auto &t : nb) {
                if (t[0] < 0 || t[1] < 0 || t[2] < 0 || t[0] >= nx || t[1] >= ny || t[2] >= nz) continue;
                const long long r = t[0] + (long long)nx * (t[1] + (long long)ny * t[2]);
                if (m[r] && comp[r] < 0) {
                    comp[r] = nc;
                    queue.push_back(r);
                }
            }
        }
        std::sort(queue.begin(), queue.end());
        for (long long r : queue) P.order.push_back((int)r);
        P.comp_count.push_back((long long)queue.size());
        ++nc;
    }
    const long long n_heart = std::count_if(s->mask.begin(), s->mask.end(), [](uint8_t c) { return c != 0; });
    if (n_heart == 0) return fail(s, EP_EINVAL, "mask has no tissue voxel");
    P.chunks.clear();
    P.comp_chunk0.assign(nc + 1, 0);
    long long pos = 0;
    for (int c = 0; c < nc; ++c) {
        P.comp_chunk0[c] = (int)P.chunks.size();
        const long long end = pos + P.comp_count[c];
        for (long long st = pos; st < end; st += kChunk)
            P.chunks.push_back(Chunk{(int)st, (int)std::min<long long>(st + kChunk, end), c});
        pos = end;
    }
    P.comp_chunk0[nc] = (int)P.chunks.size();
    long long most = 0;
    const uint8_t *mh = s->mask.data();   // the membrane kernels' items cover the tissue
    for (int i = 0; i < 4; ++i) {
        P.segs_z[i] = build_segments(mh, nx, ny, nz, kZLens[i]);
        most = std::max<long long>(most, (long long)P.segs_z[i].size());
        if (torso) {
            P.segs_e_z[i] = build_segments(m, nx, ny, nz, kZLens[i]);
            most = std::max<long long>(most, (long long)P.segs_e_z[i].size());
        }
    }
    P.segs = build_segments(mh, nx, ny, nz, s->zseg);
    if (torso) P.segs_e = build_segments(m, nx, ny, nz, s->zseg);
    s->n_tissue = n_heart;
    s->n_domain = (long long)P.order.size();
    s->ncomp = nc;
    s->nchunk = (int)P.chunks.size();
    s->nseg = (int)P.segs.size();
    s->nseg_e = torso ? (int)P.segs_e.size() : s->nseg;
    // capacity of the item buffers: the largest item count of the z-lengths set-up and the batch use
    s->max_items = std::max<long long>(most, std::max(s->nseg, s->nseg_e));
    footprint(s, s->d.precision == EP_FP64 ? sizeof(double) : sizeof(float), &s->fp_resident, &s->fp_peak);
    P.done = true;
    return EP_OK;
}


template <typename real>
Inst<real> make_inst(const ep_sim *s);
template <typename real>
Inst<real> make_elliptic_inst(const ep_sim *s);
int stencil_blocks(const ep_sim *s);

// Extreme eigenvalues of the symmetric tridiagonal (a, b) by Sturm bisection:
// the number of eigenvalues below x is the number of negative pivots of T - x I.
static int sturm_count(const std::vector<double> &a, const std::vector<double> &b, double x)
{
    int neg = 0;
    double d = 1.0;
    for (size_t i = 0; i < a.size(); ++i) {
        d = a[i] - x - (i ? b[i] * b[i] / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++neg;
    }
    return neg;
}

static double tridiag_eig(const std::vector<double> &a, const std::vector<double> &b, int which)
{
    double lo = 1e300, hi = -1e300;   // Gershgorin interval
    for (size_t i = 0; i < a.size(); ++i) {
        const double r = (i ? std::fabs(b[i]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i + 1]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    const int target = which == 0 ? 1 : (int)a.size();   // eigenvalue index (1-based, ascending)
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(a, b, mid) >= target) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Interval [lmin, lmax] of the eigenvalues of D^-1 A (A the elliptic operator,
// D its diagonal as the sweeps use it) for the Chebyshev semi-iteration:
// kLanczosSteps steps of the Lanczos process for D^-1 A in the D inner product
// (where it is self-adjoint; the same tridiagonal as symmetric Lanczos on
// D^-1/2 A D^-1/2), all on the device -- A applied by the library's operator
// kernel, FP64 inner products, the null space (constants on each component)
// D-orthogonally projected out at every step.  The host reads the tridiagonal
// once; the smallest Ritz value is scaled by 0.8 (Ritz values approach it from
// above) and the largest by 1.05.  v, vprev, w, t: n values each; lz: the
// scalars, then two partial sums per reduction chunk.
template <typename real>
ep_status estimate_cheb_interval(ep_sim *s, real *v, real *vprev, real *w, real *t, double *lz)
{
    const long long n = s->n, nt = s->n_domain;
    if (nt == 0 || s->nchunk == 0) return fail(s, EP_EINVAL, "Chebyshev interval: no tissue");
    cudaStream_t st = s->stream;
    Inst<real> I = make_elliptic_inst<real>(s);   // the domain's records (diagonal) and work items
    I.partials = lz + kLanczosScalars;
    const double sT = s->p.sig_iT + s->p.sig_eT, sL = s->p.sig_iL + s->p.sig_eL;
    ApplyIO<real> io;
    io.u = v;
    io.out = t;
    io.sT = (real)sT;
    io.dS = (real)(sL - sT);
    const int gt = grid_for(nt, kRedThreads), gc = s->nchunk, gs = std::max(1, I.nseg);
    const bool torso = !s->torso.empty();
    CK(cudaMemsetAsync(lz, 0, sizeof(double) * kLanczosScalars, st));
    k_fill<real><<<grid_for(n, 256), 256, 0, st>>>(v, n, real(0));
    k_fill<real><<<grid_for(n, 256), 256, 0, st>>>(vprev, n, real(0));
    k_lz_start<real><<<gt, kRedThreads, 0, st>>>(I, nt, w);
    k_lz_proj<real><<<gc, kRedThreads, 0, st>>>(I, v, w, lz, 0);
    k_lz_norm<real><<<gc, kRedThreads, 0, st>>>(I, w, lz, -1);
    k_lz_next<real><<<gt, kRedThreads, 0, st>>>(I, nt, v, vprev, w, lz);
    for (int j = 0; j < kLanczosSteps; ++j) {
        if (torso) k_stencil<real, M_APPLY_BATH><<<gs, kThreads, kSmemBytes<real, M_APPLY_BATH>, st>>>(I, io);
        else k_stencil<real, M_APPLY><<<gs, kThreads, kSmemBytes<real, M_APPLY>, st>>>(I, io);
        k_lz_w<real><<<gc, kRedThreads, 0, st>>>(I, t, v, vprev, w, lz);
        k_lz_proj<real><<<gc, kRedThreads, 0, st>>>(I, v, w, lz, 1);
        k_lz_norm<real><<<gc, kRedThreads, 0, st>>>(I, w, lz, j);
        k_lz_next<real><<<gt, kRedThreads, 0, st>>>(I, nt, v, vprev, w, lz);
    }
    CK(cudaGetLastError());
    std::vector<double> h(kLanczosScalars);
    CK(cudaMemcpyAsync(h.data(), lz, sizeof(double) * kLanczosScalars, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h[2] == 0.0 && h[3] == 0.0) return fail(s, EP_EINVAL, "Chebyshev interval: no coupled tissue voxels");
    std::vector<double> alpha, beta(1, 0.0);   // beta[i] couples rows i-1 and i
    for (int j = 0; j < kLanczosSteps; ++j) {
        const double a = h[2 + 2 * j], b = h[3 + 2 * j];
        alpha.push_back(a);
        if (!(b > 1e-12 * std::fabs(a))) break;   // invariant subspace: the Ritz values are exact
        if (j + 1 < kLanczosSteps) beta.push_back(b);
    }
    const double tmin = tridiag_eig(alpha, beta, 0), tmax = tridiag_eig(alpha, beta, 1);
    if (!(tmin > 0.0) || !(tmax > tmin)) return fail(s, EP_EINVAL, "Chebyshev interval: estimate failed");
    s->cheb_lmin = 0.8 * tmin;
    s->cheb_lmax = 1.05 * tmax;
    return EP_OK;
}

// Device set-up of a handle from its host plan.
template <typename real>
ep_status setup_typed(ep_sim *s)
{
    ep_status pst = plan_layout(s);
    if (pst != EP_OK) return pst;
    const int nx = s->d.nx, ny = s->d.ny, nz = s->d.nz;
    const long long n = s->n;
    const uint8_t *m = s->mask.data();
    if (n > 2147483647LL) return fail(s, EP_EINVAL, "grid too large for 32-bit voxel indices");
    // z-planes per work item on this device: the longest item (fewer halo planes) that still
    // leaves two waves of resident sweep CTAs, else 16, else 8 for small grids
    {
        int dev = 0, nsm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const long long wave = (long long)nsm * kMinBlocks;
        const bool tor = !s->torso.empty();   // with a torso the elliptic sweeps over the domain dominate
        int pick = 0;   // index into kZLens
        for (int i = 3; i >= 1; --i)
            if ((long long)(tor ? s->plan.segs_e_z[i] : s->plan.segs_z[i]).size() >= (kZLens[i] == 16 ? wave : 2 * wave)) {
                pick = i;
                break;
            }
        s->plan.segs = s->plan.segs_z[pick];
        s->nseg = (int)s->plan.segs.size();
        if (tor) s->plan.segs_e = s->plan.segs_e_z[pick];
        s->nseg_e = tor ? (int)s->plan.segs_e.size() : s->nseg;
        s->nseg_far = tor ? partition_far(s->plan.segs_e, s->mask.data(), s->d.nx, s->d.ny, s->d.nz) : 0;
        s->zseg = kZLens[pick];
    }
    const HostPlan &P = s->plan;
    const std::vector<int> &order = P.order;
    const std::vector<Chunk> &chunks = P.chunks;
    const std::vector<int> &comp_chunk0 = P.comp_chunk0;
    const std::vector<long long> &comp_count = P.comp_count;
    const std::vector<Seg> &segs = P.segs;
    const int nc = s->ncomp;
    footprint(s, sizeof(real), &s->fp_resident, &s->fp_peak);   // the parameters are known now
    const size_t want_resident = s->fp_resident, want_peak = s->fp_peak;
    const bool ie = s->p.diffusion == EP_IMPLICIT;
    const bool torso = !s->torso.empty();

    // device buffers
    const size_t rb = sizeof(real);
    s->rsz = rb;
    s->rec = (float4 *)dalloc(s, sizeof(float4) * n);
    for (int i = 0; i < 2; ++i) {
        s->v[i] = dalloc(s, rb * n);
        s->w[i] = dalloc(s, rb * n);
        s->x[i] = dalloc(s, rb * n);
    }
    s->b = dalloc(s, rb * n);
    s->tact = dalloc(s, rb * n);
    s->segs = (Seg *)dalloc(s, sizeof(Seg) * (size_t)s->max_items);
    s->idx = (int *)dalloc(s, sizeof(int) * order.size());
    s->chunks = (Chunk *)dalloc(s, sizeof(Chunk) * chunks.size());
    s->comp_chunk0 = (int *)dalloc(s, sizeof(int) * comp_chunk0.size());
    s->comp_count = (long long *)dalloc(s, sizeof(long long) * comp_count.size());
    s->means = (double *)dalloc(s, sizeof(double) * nc);
    s->partials = (double *)dalloc(s, sizeof(double) * (size_t)partial_slots(s));
    s->ctl = (Ctl *)dalloc(s, sizeof(Ctl));
    if (ie) {
        s->ie_x = dalloc(s, rb * n);
        s->ie_inv = dalloc(s, rb * n);
        if (!s->ie_x || !s->ie_inv) return fail(s, EP_ENOMEM, "device allocation failed");
    }
    s->x2 = nullptr;
    if (solve_eform(s, rb)) {
        s->x2 = dalloc(s, rb * n);
        if (!s->x2) return fail(s, EP_ENOMEM, "device allocation failed");
    }
    s->rec_e = s->rec;
    s->segs_e = s->segs;
    if (torso) {
        s->rec_e = (float4 *)dalloc(s, sizeof(float4) * n);
        s->segs_e = (Seg *)dalloc(s, sizeof(Seg) * (size_t)s->max_items);
        if (!s->rec_e || !s->segs_e) return fail(s, EP_ENOMEM, "device allocation failed");
    }
    if (s->ecg_q[0] >= 0) {
        s->ecg = (double *)dalloc(s, sizeof(double) * 3 * (size_t)s->ecg_cap);
        if (!s->ecg) return fail(s, EP_ENOMEM, "device allocation failed");
    }
    void *tmp_fib = dalloc(s, sizeof(float) * 3 * n);
    void *tmp_mask = dalloc(s, n);
    void *tmp_rec = dalloc(s, sizeof(float4) * n);
    void *tmp_lz = lanczos_bytes(s) ? dalloc(s, lanczos_bytes(s)) : nullptr;
    if (lanczos_bytes(s) && !tmp_lz) return fail(s, EP_ENOMEM, "device allocation failed");
    void *tmp_torso = torso ? dalloc(s, n) : nullptr;
    if (torso && !tmp_torso) return fail(s, EP_ENOMEM, "device allocation failed");
    const void *all[] = {s->rec, s->v[0], s->v[1], s->w[0], s->w[1], s->x[0], s->x[1], s->b, s->tact, s->segs,
                         s->idx, s->chunks, s->comp_chunk0, s->comp_count, s->means, s->partials, s->ctl,
                         tmp_fib, tmp_mask, tmp_rec};
    for (const void *p : all)
        if (!p) return fail(s, EP_ENOMEM, "device allocation failed");
    if (s->dev_bytes != want_peak) return fail(s, EP_ECUDA, "internal: set-up allocations differ from the footprint");
    cudaStream_t st = s->stream;
    CK(cudaMemcpyAsync(s->segs, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->idx, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->chunks, chunks.data(), sizeof(Chunk) * chunks.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->comp_chunk0, comp_chunk0.data(), sizeof(int) * comp_chunk0.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(s->comp_count, comp_count.data(), sizeof(long long) * comp_count.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(tmp_mask, m, n, cudaMemcpyHostToDevice, st));
    if (s->fib.empty()) CK(cudaMemsetAsync(tmp_fib, 0, sizeof(float) * 3 * n, st));
    else CK(cudaMemcpyAsync(tmp_fib, s->fib.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
    k_build_records<<<grid_for(n, 256), 256, 0, st>>>(nx, ny, nz, (const float *)tmp_fib, (const uint8_t *)tmp_mask,
                                                      nullptr, (float4 *)tmp_rec);
    // Jacobi diagonal of the elliptic operator L_i + L_e (conductivities add)
    const double sL = s->p.sig_iL + s->p.sig_eL, sT = s->p.sig_iT + s->p.sig_eT;
    k_build_diag<<<grid_for(n, 128), 128, 0, st>>>(nx, ny, nz, sT, sL - sT, 0.0, (const float4 *)tmp_rec, s->rec);
    CK(cudaGetLastError());
    if (torso) {   // the domain's records: torso voxels tagged, the diagonal with the torso term
        CK(cudaMemcpyAsync(tmp_torso, s->torso.data(), n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(s->segs_e, s->plan.segs_e.data(), sizeof(Seg) * s->plan.segs_e.size(), cudaMemcpyHostToDevice, st));
        k_build_records<<<grid_for(n, 256), 256, 0, st>>>(nx, ny, nz, (const float *)tmp_fib, (const uint8_t *)tmp_mask,
                                                          (const uint8_t *)tmp_torso, (float4 *)tmp_rec);
        k_build_diag<<<grid_for(n, 128), 128, 0, st>>>(nx, ny, nz, sT, sL - sT, s->sig_o, (const float4 *)tmp_rec,
                                                       s->rec_e);
        CK(cudaGetLastError());
    }
    if (ie) {   // implicit diffusion: 1 / (1 + a D_i) for the intracellular operator, second iterate
        const double C = 1.0 / (8.0 * s->d.dx_mm * s->d.dx_mm);
        const double fac = s->d.model == EP_MONO ? s->p.lambda / (1.0 + s->p.lambda) : 1.0;
        const double aC = s->p.dt_ms / s->p.K * fac * C;
        k_build_ie_diag<real><<<grid_for(n, 128), 128, 0, st>>>(nx, ny, nz, s->p.sig_iT, s->p.sig_iL - s->p.sig_iT,
                                                                 aC, s->rec, (real *)s->ie_inv);
        k_fill<real><<<grid_for(n, 256), 256, 0, st>>>((real *)s->ie_x, n, real(0));
        CK(cudaGetLastError());
    }
    // the spectrum of D^-1 A: for the Chebyshev solver, and for damped Jacobi with estimated damping
    if (needs_spectrum(s) && s->d.model == EP_BI) {
        if (s->p.cheb_lmin > 0.0) {
            s->cheb_lmin = s->p.cheb_lmin;
            s->cheb_lmax = s->p.cheb_lmax;
        } else {   // the state buffers serve as the Lanczos vectors before the rest state is written
            CK(cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), st));   // the reductions' arrival counter
            ep_status es = estimate_cheb_interval<real>(s, (real *)s->v[0], (real *)s->v[1], (real *)s->w[0],
                                                        (real *)s->w[1], (double *)tmp_lz);
            if (es != EP_OK) return es;
        }
        // estimated damping: omega lambda_max = 1.9 / 1.05 on the largest Ritz value (below 2 with room
        // for the estimate's error), the fastest contraction of the slow modes that stays stable
        if (s->p.jacobi_omega < 0.0) s->omega = std::min(1.0, 1.9 / s->cheb_lmax);
    }
    // rest state
    for (int i = 0; i < 2; ++i) {
        k_fill<real><<<grid_for(n, 256), 256, 0, st>>>((real *)s->v[i], n, real(0));
        k_fill<real><<<grid_for(n, 256), 256, 0, st>>>((real *)s->w[i], n, real(1));
        k_fill<real><<<grid_for(n, 256), 256, 0, st>>>((real *)s->x[i], n, real(0));
    }
    k_fill<real><<<grid_for(n, 256), 256, 0, st>>>((real *)s->b, n, real(0));
    if (s->x2) k_fill<real><<<grid_for(n, 256), 256, 0, st>>>((real *)s->x2, n, real(0));
    k_fill<real><<<grid_for(n, 256), 256, 0, st>>>((real *)s->tact, n, real(-1));
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(s->ctl, 0, sizeof(Ctl), st));
    CK(cudaStreamSynchronize(st));
    // free the set-up temporaries
    for (void *t : {tmp_fib, tmp_mask, tmp_rec, tmp_lz, tmp_torso}) {
        if (!t) continue;
        auto it = std::find(s->allocs.begin(), s->allocs.end(), t);
        if (it != s->allocs.end()) {
            if (s->d.dev_alloc && s->d.dev_free) s->d.dev_free(t, s->d.alloc_ctx);
            else cudaFree(t);
            s->allocs.erase(it);
        }
    }
    s->dev_bytes = want_resident;
    // the host plan is not needed once on the device (counts stay in the handle)
    s->plan.order = std::vector<int>();
    s->plan.comp_count = std::vector<long long>();
    s->plan.chunks = std::vector<Chunk>();
    s->plan.comp_chunk0 = std::vector<int>();
    s->plan.segs = std::vector<Seg>();
    s->plan.segs_e = std::vector<Seg>();
    for (auto &v : s->plan.segs_z) v = std::vector<Seg>();
    for (auto &v : s->plan.segs_e_z) v = std::vector<Seg>();
    CK(cudaMallocHost((void **)&s->ctl_host, 2 * sizeof(Ctl)));
    std::memset(s->ctl_host, 0, 2 * sizeof(Ctl));
    CK(cudaEventCreateWithFlags(&s->ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&s->ev[1], cudaEventDisableTiming));

    return EP_OK;
}

// Descriptor of the elliptic sweeps: the work items and records of the domain
// (tissue + torso); the tissue descriptor without a torso.
template <typename real>
Inst<real> make_elliptic_inst(const ep_sim *s)
{
    Inst<real> I = make_inst<real>(s);
    I.segs = s->segs_e;
    I.nseg = s->nseg_e;
    I.rec = s->rec_e;
    return I;
}

// Descriptor of this handle for the kernels.
template <typename real>
Inst<real> make_inst(const ep_sim *s)
{
    Inst<real> I;
    std::memset(&I, 0, sizeof(I));
    I.nx = s->d.nx;
    I.ny = s->d.ny;
    I.nz = s->d.nz;
    I.model = s->d.model == EP_MONO ? MODEL_MONO : MODEL_BI;
    I.nseg = s->nseg;
    I.nchunk = s->nchunk;
    I.ncomp = s->ncomp;
    I.check_every = s->p.check_every;
    I.max_iter = s->p.max_iter;
    I.segs = s->segs;
    I.rec = s->rec;
    for (int i = 0; i < 2; ++i) {
        I.v[i] = (real *)s->v[i];
        I.w[i] = (real *)s->w[i];
    }
    I.x0 = (real *)s->x[0];
    I.x1 = (real *)s->x[1];
    I.b = (real *)s->b;
    I.tact = (real *)s->tact;
    I.idx = s->idx;
    I.chunks = s->chunks;
    I.comp_chunk0 = s->comp_chunk0;
    I.comp_count = s->comp_count;
    I.means = s->means;
    I.partials = s->partials;
    I.ctl = s->ctl;
    I.diffusion = s->p.diffusion;
    I.pad2 = 0;
    I.ie_x = (real *)s->ie_x;
    I.ie_inv = (const real *)s->ie_inv;
    I.x2 = (real *)s->x2;
    const double C = 1.0 / (8.0 * s->d.dx_mm * s->d.dx_mm);
    const double sLie = s->p.sig_iL + s->p.sig_eL, sTie = s->p.sig_iT + s->p.sig_eT;
    const double fac = s->d.model == EP_MONO ? s->p.lambda / (1.0 + s->p.lambda) : 1.0;
    I.sTi = (real)s->p.sig_iT;
    I.dSi = (real)(s->p.sig_iL - s->p.sig_iT);
    I.sTie = (real)sTie;
    I.dSie = (real)(sLie - sTie);
    I.C = (real)C;
    I.coef_par = (real)(s->p.dt_ms / s->p.K * fac);
    I.coef_jac = (real)(s->omega / C);
    I.alpha_ie = (real)(s->p.dt_ms / s->p.K * fac);
    I.solver = s->p.solver == EP_SOLVER_CHEBYSHEV && s->cheb_lmax > 0.0 ? 1
               : s->p.solver == EP_SOLVER_GAUSS_SEIDEL && s->d.model == EP_BI ? 2 : 0;
    I.pad3 = 0;
    I.cheb_tau_c = real(0);
    I.cheb_rho = I.cheb_theta = 0.0;
    I.eform = I.solver != 2 && s->x2 ? 1 : 0;
    I.pad5 = 0;
    if (I.solver) {
        const double lo = s->cheb_lmin, hi = s->cheb_lmax;
        const double rho = (hi - lo) / (hi + lo);
        I.cheb_tau_c = (real)(2.0 / (lo + hi) / C);
        I.cheb_rho = rho;
        I.cheb_theta = std::acosh(1.0 / rho);
    }
    I.torso = s->torso.empty() ? 0 : 1;
    I.pad4 = 0;
    I.sig_o = (real)(s->torso.empty() ? 0.0 : s->sig_o);
    I.dt = (real)s->p.dt_ms;
    I.inv_tin = (real)(1.0 / s->p.tau_in);
    I.inv_tout = (real)(1.0 / s->p.tau_out);
    I.inv_topen = (real)(1.0 / s->p.tau_open);
    I.inv_tclose = (real)(1.0 / s->p.tau_close);
    I.vgate = (real)s->p.v_gate;
    I.dt_d = s->p.dt_ms;
    I.rel_tol2 = s->p.rel_tol * s->p.rel_tol;
    I.div_factor = kDivFactor;
    I.stim.n = 0;
    for (const StimDef &d : s->stims) {
        StimBox &b = I.stim.box[I.stim.n++];
        for (int i = 0; i < 3; ++i) {
            b.lo[i] = d.lo[i];
            b.hi[i] = d.hi[i];
        }
        b.t0 = d.t0;
        b.t1 = d.t0 + d.dur;   // the same double expression as t_start + dur
        b.amp = d.amp;
    }
    return I;
}

template <typename real>
ApplyIO<real> no_io()
{
    ApplyIO<real> io;
    std::memset(&io, 0, sizeof(io));
    return io;
}

// One sweep of a solve on stream q: a sweep kernel over descriptor I (one CTA
// per work item of I), or, for a torso handle whose items split, the
// single-term kernel over the items far from the tissue and the two-term one
// over the rest.
template <typename real, int MODE>
struct OneSweep {
    Inst<real> I;
    void operator()(cudaStream_t q) const
    {
        k_stencil<real, MODE><<<std::max(1, I.nseg), kThreads, kSmemBytes<real, MODE>, q>>>(I, no_io<real>());
    }
};
template <typename real, int MODE_FAR, int MODE_NEAR>
struct SplitSweep {
    Inst<real> far, near;   // far.nseg or near.nseg may be 0
    void operator()(cudaStream_t q) const
    {
        if (far.nseg > 0) k_stencil<real, MODE_FAR><<<far.nseg, kThreads, kSmemBytes<real, MODE_FAR>, q>>>(far, no_io<real>());
        if (near.nseg > 0) k_stencil<real, MODE_NEAR><<<near.nseg, kThreads, kSmemBytes<real, MODE_NEAR>, q>>>(near, no_io<real>());
    }
};

// A CUDA graph of kSweepChunk sweeps of one solve.
template <typename Sweep>
ep_status build_sweep_graph(ep_sim *s, const Sweep &sweep, cudaGraphExec_t *out)
{
    if (*out) return EP_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < kSweepChunk; ++i) sweep(s->stream);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (e != cudaSuccess) return fail(s, EP_ECUDA, std::string("sweep graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(s, EP_ECUDA, std::string("sweep graph instantiate: ") + cudaGetErrorString(e));
    }
    return EP_OK;
}

// Queues the sweeps of one solve in graph chunks with one chunk of look-ahead:
// the host reads the control block one chunk behind, so the GPU never waits
// for it.  At most max_iter sweeps (per_sweep launches each) do work; the
// launch after them marks a capped solve done.  Returns the launches queued in
// *queued_out.
template <typename Sweep>
ep_status run_sweeps(ep_sim *s, const Sweep &sweep, cudaGraphExec_t *graph, long long *queued_out, int per_sweep = 1)
{
    cudaStream_t st = s->stream;
    if (!s->noalloc_call) {
        ep_status gs = build_sweep_graph(s, sweep, graph);
        if (gs != EP_OK) return gs;
    }
    const long long limit = (long long)per_sweep * s->p.max_iter + 1;
    long long queued = 0;
    for (int c = 0;; ++c) {
        if (!s->noalloc_call && queued + kSweepChunk <= limit) {
            CK(cudaGraphLaunch(*graph, st));
            queued += kSweepChunk;
        } else {
            const long long stop = std::min(limit, queued + (long long)kSweepChunk);
            for (; queued < stop; ++queued) sweep(st);
            CK(cudaGetLastError());
        }
        CK(cudaMemcpyAsync(&s->ctl_host[c & 1], s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(s->ev[c & 1], st));
        if (queued >= limit) {   // everything up to the cap is queued; the last launch marks done
            CK(cudaEventSynchronize(s->ev[c & 1]));
            break;
        }
        if (c >= 1) {            // one chunk of look-ahead keeps the GPU busy while the host checks
            CK(cudaEventSynchronize(s->ev[(c - 1) & 1]));
            if (s->ctl_host[(c - 1) & 1].done) break;
        }
    }
    *queued_out = queued;
    return EP_OK;
}

}  // namespace

namespace {

template <typename F>
cudaError_t allow_smem(F *fn, size_t bytes)
{
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
}

template <typename real, int... MODES>
cudaError_t allow_stencil(std::integer_sequence<int, MODES...>)
{
    cudaError_t e = cudaSuccess;
    ((e = e == cudaSuccess ? allow_smem(k_stencil<real, MODES>, kSmemBytes<real, MODES>) : e), ...);
    return e;
}

template <int... MODES>
cudaError_t allow_stencil_batch(std::integer_sequence<int, MODES...>)
{
    cudaError_t e = cudaSuccess;
    ((e = e == cudaSuccess ? allow_smem(k_stencil_batch<float, MODES>, kSmemBytes<float, MODES>) : e), ...);
    return e;
}

template <int... MODES>
cudaError_t allow_stencil_active(std::integer_sequence<int, MODES...>)
{
    cudaError_t e = cudaSuccess;
    ((e = e == cudaSuccess ? allow_smem(k_stencil_active<float, MODES>, kSmemBytes<float, MODES>) : e), ...);
    return e;
}

}  // namespace

// The stencil kernels take their shared memory dynamically (with the cp.async
// rings and fp32 records several exceed the 48 KB of static shared memory):
// raise every instance's limit on the current device.  Idempotent; called at
// every set-up, so it follows the device (and context) the handle runs on.
ep_status configure_kernels(ep_sim *s)
{
    using Modes = std::integer_sequence<int, M_APPLY, M_RHS, M_PAR_MONO, M_PAR_BI, M_JAC, M_IE_RHS, M_IE, M_JAC_BATH,
                                        M_APPLY_BATH, M_JAC_CHEB, M_JAC_BATH_CHEB, M_JAC_GS>;
    cudaError_t e = allow_stencil<float>(Modes{});
    if (e == cudaSuccess) e = allow_stencil<double>(Modes{});
    if (e == cudaSuccess)
        e = allow_stencil_batch(std::integer_sequence<int, M_PAR_MONO, M_PAR_BI, M_RHS, M_JAC, M_JAC_CHEB>{});
    if (e == cudaSuccess) e = allow_stencil_active(std::integer_sequence<int, M_JAC, M_JAC_CHEB>{});
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(s, EP_ECUDA, std::string("cudaFuncSetAttribute(shared memory): ") + cudaGetErrorString(e));
    }
    return EP_OK;
}

ep_status ensure_ready(ep_sim *s)
{
    if (s->ready) return EP_OK;
    if (!s->have_mask) return fail(s, EP_ESTATE, "ep_set_mask must be called before stepping");
    if (!s->have_params) return fail(s, EP_ESTATE, "ep_set_params must be called before stepping");
    if (!s->stream) {
        // a non-blocking private stream: CUDA-graph capture needs a stream other than the legacy one
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->stream = nullptr;
            return fail(s, EP_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
        }
        s->own_stream = true;
    }
    if (!s->torso.empty() && (s->d.model != EP_BI || s->p.diffusion != EP_EXPLICIT))
        return fail(s, EP_EINVAL, "a torso needs the bidomain model with explicit diffusion");
    if (s->ecg_q[0] >= 0) {
        if (s->d.model != EP_BI) return fail(s, EP_EINVAL, "the ECG needs the bidomain model (it reads v_e)");
        for (int e = 0; e < 3; ++e) {
            const int q = s->ecg_q[e];
            if (!s->mask[q] && (s->torso.empty() || !s->torso[q]))
                return fail(s, EP_EINVAL, "ECG electrodes must lie on tissue or torso voxels");
        }
    }
    const double sL = s->p.sig_iL + s->p.sig_eL, sT = s->p.sig_iT + s->p.sig_eT;
    s->omega = s->p.jacobi_omega > 0.0 ? s->p.jacobi_omega : std::min(1.0, 1.8 * (sL + 2.0 * sT) / (8.0 * sL));
    if (s->p.solver == EP_SOLVER_GAUSS_SEIDEL) {   // SOR factor: given, else Gauss-Seidel
        if (!s->torso.empty()) return fail(s, EP_EINVAL, "the Gauss-Seidel solve does not take a torso");
        s->omega = s->p.jacobi_omega > 0.0 ? s->p.jacobi_omega : 1.0;
    }
    ep_status cs = configure_kernels(s);
    if (cs != EP_OK) return cs;
    ep_status st = s->d.precision == EP_FP64 ? setup_typed<double>(s) : setup_typed<float>(s);
    if (st != EP_OK) {
        dfree_all(s);
        return st;
    }
    s->ready = true;
    return EP_OK;
}

namespace {

// Writes the device step counter (the state of step n lives in buffers n & 1).
ep_status set_device_step(ep_sim *s, long long step)
{
    CK(cudaMemcpyAsync((char *)s->ctl + offsetof(Ctl, step), &step, sizeof(step), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->step = step;
    return EP_OK;
}

template <typename real>
ep_status solve_elliptic(ep_sim *s, const Inst<real> &I, int &iters, double &relres, int &conv, int &flags)
{
    cudaStream_t st = s->stream;
    const ApplyIO<real> io = no_io<real>();
    // b = -L_i v, zero mean per component, ||b|| and a fresh solve in ctl
    k_stencil<real, M_RHS><<<stencil_blocks(s), kThreads, kSmemBytes<real, M_RHS>, st>>>(I, io);
    k_comp_mean<real><<<s->nchunk, kRedThreads, 0, st>>>(I, (int)RED_B);
    k_comp_subtract<real><<<s->nchunk, kRedThreads, 0, st>>>(I);
    CK(cudaGetLastError());
    // sweeps, queued in graph chunks, one chunk of look-ahead
    if (s->prof_on) CK(cudaEventRecord(s->pev[2], st));
    long long queued = 0;
    ep_status rs = EP_OK;
    const bool cheb = I.solver == 1;   // the sweep instance matches the handle's solver
    if (I.solver == 2) {   // eight colour passes a sweep
        rs = run_sweeps(s, OneSweep<real, M_JAC_GS>{I}, &s->sweep_graph, &queued, 8);
    } else if (s->torso.empty()) {
        rs = cheb ? run_sweeps(s, OneSweep<real, M_JAC_CHEB>{I}, &s->sweep_graph, &queued)
                  : run_sweeps(s, OneSweep<real, M_JAC>{I}, &s->sweep_graph, &queued);
    } else {   // tissue + torso: the domain's items and records, split by distance from the tissue
        const Inst<real> Ie = make_elliptic_inst<real>(s);
        Inst<real> far = Ie, near = Ie;
        far.nseg = s->nseg_far;                 // items far from the tissue come first
        far.nitems_all = near.nitems_all = s->nseg_e;
        far.sTie = (real)s->sig_o;              // there the operator is the torso term alone:
        far.dSie = real(0);                     // the plain one with sigma = sig_o I
        near.segs = s->segs_e + s->nseg_far;
        near.nseg = s->nseg_e - s->nseg_far;
        near.item0 = s->nseg_far;
        rs = cheb ? run_sweeps(s, SplitSweep<real, M_JAC_CHEB, M_JAC_BATH_CHEB>{far, near}, &s->sweep_graph, &queued)
                  : run_sweeps(s, SplitSweep<real, M_JAC, M_JAC_BATH>{far, near}, &s->sweep_graph, &queued);
    }
    if (rs != EP_OK) return rs;
    if (s->prof_on) {
        CK(cudaEventRecord(s->pev[3], st));
        s->prof.sweep_launches += queued;
        s->prof.other_launches += 5;   // RHS, 2 reductions + subtract, projection
    }
    // reference potential: subtract each component's mean of the final iterate
    k_comp_mean<real><<<s->nchunk, kRedThreads, 0, st>>>(I, (int)RED_X_FINAL);
    k_project<real><<<s->nchunk, kRedThreads, 0, st>>>(I);
    if (s->ecg_q[0] >= 0) {   // electrode potentials of this step
        k_ecg_record<real><<<1, 32, 0, st>>>(I.x0, s->ecg_q[0], s->ecg_q[1], s->ecg_q[2], s->ecg, s->ecg_n);
        if (s->ecg_n == 0) s->ecg_t0 = (double)(s->step + 1) * s->p.dt_ms;
        ++s->ecg_n;
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&s->ctl_host[0], s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const Ctl &h = s->ctl_host[0];
    if (s->prof_on) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, s->pev[2], s->pev[3]));
        s->prof.sweep_ms += ms;
        s->prof.sweeps += h.iters;
    }
    iters = h.iters;
    relres = h.bnorm2 > 0.0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
    conv = h.converged;
    flags = (h.nonfinite ? 1 : 0) | (h.diverged ? 2 : 0);
    return EP_OK;
}

template <typename real>
ep_status step_typed(ep_sim *s, int n_steps, ep_step_stats *stats)
{
    cudaStream_t st = s->stream;
    ep_status ret = EP_OK;
    int last_iters = 0, all_conv = 1;
    double last_rr = 0.0;
    long long total = 0;
    const Inst<real> I = make_inst<real>(s);
    const ApplyIO<real> io = no_io<real>();
    const bool ie = s->p.diffusion == EP_IMPLICIT;
    {   // the flags of this call (non-finite, diverged, not converged) start clear
        static_assert(offsetof(Ctl, diverged) == offsetof(Ctl, nonfinite) + sizeof(int) &&
                          offsetof(Ctl, noconv) == offsetof(Ctl, diverged) + sizeof(int),
                      "the call's flags are adjacent");
        const int zero[3] = {0, 0, 0};
        CK(cudaMemcpyAsync((char *)s->ctl + offsetof(Ctl, nonfinite), zero, sizeof(zero), cudaMemcpyHostToDevice, st));
    }
    for (int it = 0; it < n_steps; ++it) {
        const double sweep_ms0 = s->prof.sweep_ms;
        if (s->prof_on) CK(cudaEventRecord(s->pev[0], st));
        if (ie) {
            // implicit Euler (Eq. iejac1): reaction and right-hand side f, ||f||, Jacobi sweeps
            // from v* to rel_tol, then the final iterate, activation times and the flags
            const int gt = grid_for(s->n_tissue, kRedThreads);
            if (s->d.model == EP_MONO) k_ie_react<real><<<gt, kRedThreads, 0, st>>>(I);
            else k_stencil<real, M_IE_RHS><<<stencil_blocks(s), kThreads, kSmemBytes<real, M_IE_RHS>, st>>>(I, io);
            k_ie_start<real><<<s->nchunk, kRedThreads, 0, st>>>(I);
            CK(cudaGetLastError());
            if (s->prof_on) CK(cudaEventRecord(s->pev[4], st));
            long long queued = 0;
            ep_status e = run_sweeps(s, OneSweep<real, M_IE>{I}, &s->ie_graph, &queued);
            if (e != EP_OK) return e;
            if (s->prof_on) {
                CK(cudaEventRecord(s->pev[5], st));
                s->prof.other_launches += 3 + queued;
            }
            k_ie_finish<real><<<gt, kRedThreads, 0, st>>>(I);
        } else {
            // reaction + diffusion: reads v, w of step n (buffer n & 1), writes buffer (n + 1) & 1
            if (s->d.model == EP_MONO) k_stencil<real, M_PAR_MONO><<<stencil_blocks(s), kThreads, kSmemBytes<real, M_PAR_MONO>, st>>>(I, io);
            else k_stencil<real, M_PAR_BI><<<stencil_blocks(s), kThreads, kSmemBytes<real, M_PAR_BI>, st>>>(I, io);
        }
        CK(cudaGetLastError());
        if (s->d.model == EP_BI) {
            int iters = 0, conv = 0, flags = 0;
            double rr = 0.0;
            ep_status e = solve_elliptic<real>(s, I, iters, rr, conv, flags);
            if (e != EP_OK) return e;
            last_iters = iters;
            last_rr = rr;
            total += iters;
            if (!conv) all_conv = 0;
            if (flags & 1) ret = EP_ENONFINITE;
            else if (!conv && ret == EP_OK) ret = EP_ENOCONV;
        }
        k_end_step<real><<<1, 32, 0, st>>>(nullptr, 0, I);
        CK(cudaGetLastError());
        if (s->prof_on) {
            CK(cudaEventRecord(s->pev[1], st));
            CK(cudaEventSynchronize(s->pev[1]));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, s->pev[0], s->pev[1]));
            s->prof.other_ms += ms - (s->prof.sweep_ms - sweep_ms0);
            s->prof.other_launches += 2;
            s->prof.steps += 1;
            if (ie) {
                CK(cudaEventElapsedTime(&ms, s->pev[4], s->pev[5]));
                s->prof.ie_sweep_ms += ms;
            }
        }
        s->step++;
    }
    CK(cudaMemcpyAsync(&s->ctl_host[1], s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const Ctl &h = s->ctl_host[1];
    if (h.nonfinite) ret = EP_ENONFINITE;
    else if (h.noconv && ret == EP_OK) ret = EP_ENOCONV;   // an implicit solve hit its cap or diverged
    const long long ie_calls = h.ie_total - s->ie_seen;
    s->ie_seen = h.ie_total;
    if (s->prof_on) s->prof.ie_sweeps += ie_calls;
    if (stats) {
        stats->iters = last_iters;
        stats->rel_res = last_rr;
        stats->converged = all_conv && !h.noconv;
        stats->total_iters = total;
        stats->step = s->step;
        stats->ie_total_iters = ie_calls;
    }
    if (ret == EP_ENOCONV) s->err = "a solve reached max_iter or diverged";
    if (ret == EP_ENONFINITE) s->err = "non-finite value in the state";
    return ret;
}

template <typename real>
ep_status read_typed(ep_sim *s, int field, double *out)
{
    const void *src = nullptr;
    switch (field) {
    case EP_VM_MV: case EP_V: src = s->v[s->step & 1]; break;
    case EP_W: src = s->w[s->step & 1]; break;
    case EP_VE_MV: case EP_VE: src = s->x[0]; break;
    case EP_TACT: src = s->tact; break;
    default: return fail(s, EP_EINVAL, "unknown field");
    }
    std::vector<real> h(s->n);
    CK(cudaMemcpyAsync(h.data(), src, sizeof(real) * s->n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (long long q = 0; q < s->n; ++q) {
        const double v = (double)h[q];
        out[q] = field == EP_VM_MV ? 100.0 * v - 80.0 : field == EP_VE_MV ? 100.0 * v : v;
    }
    return EP_OK;
}

template <typename real>
ep_status set_state_typed(ep_sim *s, const double *v, const double *w, const double *ve)
{
    const double *src[3] = {v, w, ve};
    void *dst[3] = {s->v[s->step & 1], s->w[s->step & 1], s->x[0]};
    const double rest[3] = {0.0, 1.0, 0.0};
    const bool torso = !s->torso.empty();
    std::vector<real> h(s->n);
    for (int f = 0; f < 3; ++f) {
        if (!src[f]) continue;
        for (long long q = 0; q < s->n; ++q) {   // v, w on the tissue; v_e on tissue + torso
            const bool in = s->mask[q] || (f == 2 && torso && s->torso[q]);
            h[q] = (real)(in ? src[f][q] : rest[f]);
        }
        CK(cudaMemcpyAsync(dst[f], h.data(), sizeof(real) * s->n, cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    return EP_OK;
}

struct StateHeader {
    char magic[8];
    long long n;
    long long step;
    int precision;
    int pad;
};

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

ep_status ep_create(const ep_grid_desc *desc, ep_sim **out)
{
    if (!out) return EP_EINVAL;
    *out = nullptr;
    if (!desc) return EP_EINVAL;
    if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1 || !(desc->dx_mm > 0.0) || !std::isfinite(desc->dx_mm))
        return EP_EINVAL;
    if ((desc->model != EP_MONO && desc->model != EP_BI) || (desc->precision != EP_FP32 && desc->precision != EP_FP64))
        return EP_EINVAL;
    if ((desc->dev_alloc == nullptr) != (desc->dev_free == nullptr)) return EP_EINVAL;
    const long long n = (long long)desc->nx * desc->ny * desc->nz;
    if (n > 2147483647LL) return EP_EINVAL;
    ep_sim *s = new (std::nothrow) ep_sim();
    if (!s) return EP_ENOMEM;
    s->d = *desc;
    s->n = n;
    s->stream = (cudaStream_t)desc->cuda_stream;   // NULL: a private stream is created at set-up
    *out = s;
    return EP_OK;
}

ep_status ep_set_mask(ep_sim *s, const uint8_t *mask, size_t n)
{
    if (!s) return EP_EINVAL;
    if (s->ready) return fail(s, EP_ESTATE, "mask can only be set before the first step");
    if (!mask || (long long)n != s->n) return fail(s, EP_EINVAL, "mask must hold nx*ny*nz bytes");
    s->mask.assign(mask, mask + n);
    for (auto &c : s->mask) c = c ? 1 : 0;
    s->have_mask = true;
    s->plan = HostPlan();   // layout of the previous mask, if planned, is stale
    return EP_OK;
}

ep_status ep_set_fibres(ep_sim *s, const float *f, size_t n3)
{
    if (!s) return EP_EINVAL;
    if (s->ready) return fail(s, EP_ESTATE, "fibres can only be set before the first step");
    if (!f || (long long)n3 != 3 * s->n) return fail(s, EP_EINVAL, "fibres must hold 3*nx*ny*nz floats");
    for (size_t i = 0; i < n3; ++i)
        if (!std::isfinite(f[i]) || std::fabs(f[i]) > 4.0f) return fail(s, EP_EINVAL, "fibre components must be finite and at most 4 in magnitude");
    s->fib.assign(f, f + n3);
    return EP_OK;
}

ep_status ep_set_params(ep_sim *s, const ep_params *p)
{
    if (!s) return EP_EINVAL;
    if (s->ready) return fail(s, EP_ESTATE, "parameters can only be set before the first step");
    if (!p) return fail(s, EP_EINVAL, "null parameters");
    std::string why;
    if (!params_ok(*p, why)) return fail(s, EP_EINVAL, why);
    s->p = *p;
    s->have_params = true;
    return EP_OK;
}

ep_status ep_add_stimulus(ep_sim *s, const int lo[3], const int hi[3], double t_start_ms, double dur_ms,
                          double amp_per_ms)
{
    if (!s) return EP_EINVAL;
    if (s->ready) return fail(s, EP_ESTATE, "stimuli can only be added before the first step");
    if (!lo || !hi) return fail(s, EP_EINVAL, "null box");
    if ((int)s->stims.size() >= kMaxStim) return fail(s, EP_EINVAL, "at most 8 stimulus boxes");
    if (!std::isfinite(t_start_ms) || !std::isfinite(dur_ms) || dur_ms < 0.0 || !std::isfinite(amp_per_ms))
        return fail(s, EP_EINVAL, "stimulus times and amplitude must be finite, dur >= 0");
    StimDef d;
    for (int i = 0; i < 3; ++i) {
        d.lo[i] = lo[i];
        d.hi[i] = hi[i];
    }
    d.t0 = t_start_ms;
    d.dur = dur_ms;
    d.amp = amp_per_ms;
    s->stims.push_back(d);
    return EP_OK;
}

ep_status ep_set_state(ep_sim *s, const double *v, const double *w, const double *ve, size_t n, long long step)
{
    if (!s) return EP_EINVAL;
    if ((long long)n != s->n) return fail(s, EP_EINVAL, "state fields must hold nx*ny*nz doubles");
    if (step < 0) return fail(s, EP_EINVAL, "step must be >= 0");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    // the state of step n lives in buffers n & 1: carry the fields over when the parity
    // changes (a NULL field keeps its value), then move the counter
    if ((s->step ^ step) & 1) {
        const size_t fb = s->rsz * (size_t)s->n;
        CK(cudaMemcpyAsync(s->v[step & 1], s->v[s->step & 1], fb, cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync(s->w[step & 1], s->w[s->step & 1], fb, cudaMemcpyDeviceToDevice, s->stream));
    }
    st = set_device_step(s, step);
    if (st != EP_OK) return st;
    return s->d.precision == EP_FP64 ? set_state_typed<double>(s, v, w, ve) : set_state_typed<float>(s, v, w, ve);
}

ep_status ep_step(ep_sim *s, int n_steps, ep_step_stats *stats)
{
    if (!s) return EP_EINVAL;
    if (n_steps < 0) return fail(s, EP_EINVAL, "n_steps must be >= 0");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    if (s->ecg_q[0] >= 0 && s->ecg_n + n_steps > s->ecg_cap)
        return fail(s, EP_EBUSY, "the ECG record would overflow: read it with ep_read_ecg first");
    return s->d.precision == EP_FP64 ? step_typed<double>(s, n_steps, stats) : step_typed<float>(s, n_steps, stats);
}

ep_status ep_read(ep_sim *s, int field, void *host, size_t bytes)
{
    if (!s) return EP_EINVAL;
    if (!host || (long long)bytes != s->n * (long long)sizeof(double)) return fail(s, EP_EINVAL, "bytes must be n * 8");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    return s->d.precision == EP_FP64 ? read_typed<double>(s, field, (double *)host) : read_typed<float>(s, field, (double *)host);
}

ep_status ep_state_bytes(ep_sim *s, size_t *bytes)
{
    if (!s || !bytes) return EP_EINVAL;
    const size_t rb = s->d.precision == EP_FP64 ? 8 : 4;
    *bytes = sizeof(StateHeader) + 4 * rb * (size_t)s->n;
    return EP_OK;
}

ep_status ep_read_state(ep_sim *s, void *host, size_t bytes)
{
    size_t need = 0;
    if (ep_state_bytes(s, &need) != EP_OK) return EP_EINVAL;
    if (!host || bytes != need) return fail(s, EP_EINVAL, "state buffer size mismatch (see ep_state_bytes)");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    StateHeader h{};
    std::memcpy(h.magic, "EPSTATE1", 8);
    h.n = s->n;
    h.step = s->step;
    h.precision = s->d.precision;
    char *p = (char *)host;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    const size_t fb = s->rsz * (size_t)s->n;
    const void *src[4] = {s->v[s->step & 1], s->w[s->step & 1], s->x[0], s->tact};
    for (int f = 0; f < 4; ++f) CK(cudaMemcpyAsync(p + f * fb, src[f], fb, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return EP_OK;
}

ep_status ep_write_state(ep_sim *s, const void *host, size_t bytes)
{
    size_t need = 0;
    if (ep_state_bytes(s, &need) != EP_OK) return EP_EINVAL;
    if (!host || bytes != need) return fail(s, EP_EINVAL, "state buffer size mismatch (see ep_state_bytes)");
    StateHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (std::memcmp(h.magic, "EPSTATE1", 8) != 0 || h.n != s->n || h.precision != s->d.precision || h.step < 0)
        return fail(s, EP_EINVAL, "state blob does not match this handle");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    st = set_device_step(s, h.step);
    if (st != EP_OK) return st;
    const char *p = (const char *)host + sizeof(h);
    const size_t fb = s->rsz * (size_t)s->n;
    void *dst[4] = {s->v[s->step & 1], s->w[s->step & 1], s->x[0], s->tact};
    for (int f = 0; f < 4; ++f) CK(cudaMemcpyAsync(dst[f], p + f * fb, fb, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return EP_OK;
}

ep_status ep_apply_operator(ep_sim *s, double sig_L, double sig_T, const double *u_host, double *out_host, size_t n)
{
    if (!s) return EP_EINVAL;
    if (!u_host || !out_host || (long long)n != s->n) return fail(s, EP_EINVAL, "fields must hold nx*ny*nz doubles");
    if (!(sig_T > 0.0) || !(sig_L > 0.0) || !std::isfinite(sig_L) || !std::isfinite(sig_T))
        return fail(s, EP_EINVAL, "conductivities must be > 0");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    // b and x[1] are scratch between steps
    auto run = [&](auto tag) -> ep_status {
        using real = decltype(tag);
        std::vector<real> h(s->n);
        for (long long q = 0; q < s->n; ++q) h[q] = (real)u_host[q];
        CK(cudaMemcpyAsync(s->b, h.data(), sizeof(real) * s->n, cudaMemcpyHostToDevice, s->stream));
        k_fill<real><<<grid_for(s->n, 256), 256, 0, s->stream>>>((real *)s->x[1], s->n, real(0));
        const Inst<real> I = make_inst<real>(s);
        ApplyIO<real> io;
        io.u = (const real *)s->b;
        io.out = (real *)s->x[1];
        io.sT = (real)sig_T;
        io.dS = (real)(sig_L - sig_T);
        k_stencil<real, M_APPLY><<<stencil_blocks(s), kThreads, kSmemBytes<real, M_APPLY>, s->stream>>>(I, io);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h.data(), s->x[1], sizeof(real) * s->n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        for (long long q = 0; q < s->n; ++q) out_host[q] = (double)h[q];
        return EP_OK;
    };
    return s->d.precision == EP_FP64 ? run(double(0)) : run(float(0));
}

ep_status ep_get_info(ep_sim *s, ep_info *info)
{
    if (!s || !info) return EP_EINVAL;
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    info->n_voxels = s->n;
    info->n_tissue = s->n_tissue;
    info->n_components = s->ncomp;
    info->n_segments = s->nseg;
    info->omega = s->omega;
    info->cheb_lmin = s->cheb_lmin;
    info->cheb_lmax = s->cheb_lmax;
    info->device_bytes = s->dev_bytes;
    info->n_domain = s->n_domain;
    info->n_segments_elliptic = s->nseg_e;
    info->n_segments_far = s->nseg_far;
    return EP_OK;
}

ep_status ep_set_torso(ep_sim *s, const uint8_t *torso, size_t n, double sig_o)
{
    if (!s) return EP_EINVAL;
    if (s->ready) return fail(s, EP_ESTATE, "the torso can only be set before the first step");
    if (!torso || (long long)n != s->n) return fail(s, EP_EINVAL, "torso must hold nx*ny*nz bytes");
    if (!(sig_o > 0.0) || !std::isfinite(sig_o)) return fail(s, EP_EINVAL, "sig_o must be finite and > 0");
    s->torso.assign(torso, torso + n);
    bool any = false;
    for (auto &c : s->torso) {
        c = c ? 1 : 0;
        any = any || c;
    }
    if (!any) s->torso.clear();   // an empty torso is no torso
    s->sig_o = sig_o;
    s->plan = HostPlan();         // the domain changed
    return EP_OK;
}

ep_status ep_set_ecg(ep_sim *s, const int electrodes[9], int capacity)
{
    if (!s) return EP_EINVAL;
    if (s->ready) return fail(s, EP_ESTATE, "the ECG can only be set up before the first step");
    if (capacity == 0) {
        s->ecg_q[0] = s->ecg_q[1] = s->ecg_q[2] = -1;
        s->ecg_cap = 0;
        return EP_OK;
    }
    if (!electrodes || capacity < 0) return fail(s, EP_EINVAL, "electrodes must be given and capacity >= 0");
    int q[3];
    for (int e = 0; e < 3; ++e) {
        const int i = electrodes[3 * e], j = electrodes[3 * e + 1], k = electrodes[3 * e + 2];
        if (i < 0 || j < 0 || k < 0 || i >= s->d.nx || j >= s->d.ny || k >= s->d.nz)
            return fail(s, EP_EINVAL, "electrode outside the grid");
        q[e] = i + s->d.nx * (j + s->d.ny * k);
    }
    for (int e = 0; e < 3; ++e) s->ecg_q[e] = q[e];
    s->ecg_cap = capacity;
    s->ecg_n = 0;
    return EP_OK;
}

ep_status ep_read_ecg(ep_sim *s, ep_ecg_sample *out, int max_samples, int *n_out)
{
    if (!s || !n_out) return EP_EINVAL;
    *n_out = 0;
    if (s->ecg_q[0] < 0) return fail(s, EP_EINVAL, "no ECG set up (ep_set_ecg)");
    if (!s->ready || s->ecg_n == 0) return EP_OK;
    if (!out || max_samples < s->ecg_n) {
        *n_out = (int)s->ecg_n;
        return fail(s, EP_EINVAL, "max_samples is below the samples recorded (returned in *n_out)");
    }
    std::vector<double> h(3 * (size_t)s->ecg_n);
    CK(cudaMemcpyAsync(h.data(), s->ecg, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (long long i = 0; i < s->ecg_n; ++i) {
        ep_ecg_sample &o = out[i];
        o.t_ms = s->ecg_t0 + (double)i * s->p.dt_ms;
        const double ra = 100.0 * h[3 * i], la = 100.0 * h[3 * i + 1], ll = 100.0 * h[3 * i + 2];
        o.phi_mV[0] = ra;
        o.phi_mV[1] = la;
        o.phi_mV[2] = ll;
        // limb leads (Sec. "Electrocardiogram"): Einthoven's I, II, III and the augmented leads
        o.lead_mV[0] = la - ra;
        o.lead_mV[1] = ll - ra;
        o.lead_mV[2] = ll - la;
        o.lead_mV[3] = ra - 0.5 * (la + ll);
        o.lead_mV[4] = la - 0.5 * (ra + ll);
        o.lead_mV[5] = ll - 0.5 * (ra + la);
    }
    *n_out = (int)s->ecg_n;
    s->ecg_n = 0;
    return EP_OK;
}

ep_status ep_apply_elliptic(ep_sim *s, const double *u_host, double *out_host, size_t n)
{
    if (!s) return EP_EINVAL;
    if (!u_host || !out_host || (long long)n != s->n) return fail(s, EP_EINVAL, "fields must hold nx*ny*nz doubles");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    auto run = [&](auto tag) -> ep_status {   // b and x[1] are scratch between steps
        using real = decltype(tag);
        std::vector<real> h(s->n);
        for (long long q = 0; q < s->n; ++q) h[q] = (real)u_host[q];
        CK(cudaMemcpyAsync(s->b, h.data(), sizeof(real) * s->n, cudaMemcpyHostToDevice, s->stream));
        k_fill<real><<<grid_for(s->n, 256), 256, 0, s->stream>>>((real *)s->x[1], s->n, real(0));
        const Inst<real> I = make_elliptic_inst<real>(s);
        ApplyIO<real> io;
        io.u = (const real *)s->b;
        io.out = (real *)s->x[1];
        io.sT = (real)(s->p.sig_iT + s->p.sig_eT);
        io.dS = (real)(s->p.sig_iL + s->p.sig_eL - s->p.sig_iT - s->p.sig_eT);
        if (s->torso.empty()) k_stencil<real, M_APPLY><<<std::max(1, I.nseg), kThreads, kSmemBytes<real, M_APPLY>, s->stream>>>(I, io);
        else k_stencil<real, M_APPLY_BATH><<<std::max(1, I.nseg), kThreads, kSmemBytes<real, M_APPLY_BATH>, s->stream>>>(I, io);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h.data(), s->x[1], sizeof(real) * s->n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        for (long long q = 0; q < s->n; ++q) out_host[q] = (double)h[q];
        return EP_OK;
    };
    return s->d.precision == EP_FP64 ? run(double(0)) : run(float(0));
}

ep_status ep_footprint(ep_sim *s, size_t *resident_bytes, size_t *peak_bytes)
{
    if (!s || !resident_bytes || !peak_bytes) return EP_EINVAL;
    if (s->ready) {
        *resident_bytes = *peak_bytes = s->dev_bytes;
        return EP_OK;
    }
    const ep_status st = plan_layout(s);
    if (st != EP_OK) return st;
    *resident_bytes = s->fp_resident;
    *peak_bytes = s->fp_peak;
    return EP_OK;
}

ep_status ep_profile_enable(ep_sim *s, int on)
{
    if (!s) return EP_EINVAL;
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return st;
    for (auto &e : s->pev)
        if (!e) CK(cudaEventCreate(&e));
    s->prof = ep_profile{};
    s->prof_on = on != 0;
    return EP_OK;
}

ep_status ep_get_profile(ep_sim *s, ep_profile *prof)
{
    if (!s || !prof) return EP_EINVAL;
    *prof = s->prof;
    return EP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ep_step_noalloc: the elliptic-solve and non-finite-flag scratch of a step
// (control block, per-CTA partial sums, component means) comes from one
// file-scope device array instead of the handle's allocations.  Every device
// that loads the library holds the array until the process exits; all calls
// on a device share it, so calls that overlap on the GPU race.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoAllocMaxPartials = 32768;     // stencil work items and reduction chunks
constexpr int kNoAllocMaxComponents = 4096;    // face-connected tissue components
constexpr size_t kNoAllocCtlBytes = 256;       // control block slot
constexpr size_t kNoAllocBytes =
    kNoAllocCtlBytes + sizeof(double) * ((size_t)kNoAllocMaxComponents + (size_t)kNoAllocMaxPartials);
static_assert(sizeof(Ctl) <= kNoAllocCtlBytes, "control block must fit its slot");
constexpr int kNoAllocMaxDevices = 256;
std::mutex g_noalloc_mu;
struct NoAllocAddr {
    unsigned long long ctx = 0;   // context the address belongs to (0: unknown)
    void *addr = nullptr;
};
NoAllocAddr g_noalloc_addr[kNoAllocMaxDevices];

// Identity of the calling thread's current CUDA context, through the runtime's
// driver entry points (cuCtxGetCurrent, cuCtxGetId); 0 if it cannot be told.
// A context that is torn down and recreated (a device reset) gets a new
// identity, and with it a new address of the library's device arrays.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult(CUDAAPI *)(CUcontext *);
    using GetId = CUresult(CUDAAPI *)(CUcontext, unsigned long long *);
    static const GetCurrent get_current = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<GetCurrent>(p);
    }();
    static const GetId get_id = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<GetId>(p);
    }();
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
// Device address of the static scratch on the current device.  In host code
// the array's name is only a stand-in, so the address is looked up once per
// device and context (with that device current) and cached; a new context on
// the device (after a reset) looks it up again.  Without a context identity
// it is looked up on every call (the lookup allocates nothing).
ep_status noalloc_scratch(ep_sim *s, unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(s, EP_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(s, EP_EINVAL, "device ordinal out of range");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocAddr &slot = g_noalloc_addr[dev];
    if (!slot.addr || ctx == 0 || slot.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(s, EP_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        }
        slot.addr = p;
        slot.ctx = ctx;
    }
    *out = (unsigned char *)slot.addr;
    return EP_OK;
}
}  // namespace

extern "C" {

ep_status ep_step_noalloc(ep_sim *s, int n_steps, ep_step_stats *stats)
{
    if (!s) return EP_EINVAL;
    if (n_steps < 0) return fail(s, EP_EINVAL, "n_steps must be >= 0");
    if (!s->ready)
        return fail(s, EP_ESTATE, "ep_step_noalloc needs a handle that is already set up (call ep_step, "
                                  "ep_set_state or ep_get_info once first): set-up allocates device memory");
    if (s->ecg_q[0] >= 0 && s->ecg_n + n_steps > s->ecg_cap)
        return fail(s, EP_EBUSY, "the ECG record would overflow: read it with ep_read_ecg first");
    const long long passes = s->p.solver == EP_SOLVER_GAUSS_SEIDEL ? 8 : 1;   // partial sums per work item
    if (passes * std::max(stencil_blocks(s), s->nseg_e) > kNoAllocMaxPartials || s->nchunk > kNoAllocMaxPartials)
        return fail(s, EP_EINVAL, "grid too large for ep_step_noalloc: more than 32768 stencil work items "
                                  "(4096 with the Gauss-Seidel solve) or reduction chunks (use ep_step)");
    if (s->ncomp > kNoAllocMaxComponents)
        return fail(s, EP_EINVAL, "mask has more than 4096 tissue components: too many for ep_step_noalloc "
                                  "(use ep_step)");
    unsigned char *base = nullptr;
    ep_status st = noalloc_scratch(s, &base);
    if (st != EP_OK) return st;
    Ctl *ctl = (Ctl *)base;
    double *means = (double *)(base + kNoAllocCtlBytes);
    double *partials = means + kNoAllocMaxComponents;
    // the array keeps the previous call's contents: clear the arrival counter and the
    // flags, and carry the handle's step counter in
    CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s->stream));
    const long long step0 = s->step;
    CK(cudaMemcpyAsync((char *)ctl + offsetof(Ctl, step), &step0, sizeof(step0), cudaMemcpyHostToDevice, s->stream));
    Ctl *ctl0 = s->ctl;
    double *means0 = s->means, *partials0 = s->partials;
    s->ctl = ctl;
    s->means = means;
    s->partials = partials;
    s->noalloc_call = true;
    const long long ie_seen0 = s->ie_seen;
    s->ie_seen = 0;   // the static control block counts implicit sweeps from zero
    st = s->d.precision == EP_FP64 ? step_typed<double>(s, n_steps, stats) : step_typed<float>(s, n_steps, stats);
    s->ie_seen = ie_seen0;
    s->ctl = ctl0;
    s->means = means0;
    s->partials = partials0;
    s->noalloc_call = false;
    // the handle's own control block follows the step counter
    const long long step1 = s->step;
    CK(cudaMemcpyAsync((char *)s->ctl + offsetof(Ctl, step), &step1, sizeof(step1), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return st;
}

const char *ep_last_error(const ep_sim *s)
{
    if (!s) return "null handle";
    return s->err.c_str();
}

void ep_destroy(ep_sim *s)
{
    if (!s) return;
    if (s->ready && s->stream) cudaStreamSynchronize(s->stream);
    if (s->sweep_graph) cudaGraphExecDestroy(s->sweep_graph);
    if (s->ie_graph) cudaGraphExecDestroy(s->ie_graph);
    for (auto &e : s->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : s->pev)
        if (e) cudaEventDestroy(e);
    if (s->ctl_host) cudaFreeHost(s->ctl_host);
    dfree_all(s);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"

// ===========================================================================
// Batched form (config 3) and the basis of the serving loop.
// ===========================================================================
struct ep_batch {
    int max_inst = 0;
    size_t budget = 0;
    cudaStream_t stream = nullptr, side = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<ep_sim *> slot;   // nullptr = free
    int model = -1;
    // device tables: descriptors, packed stencil items, packed reduction chunks
    Inst<float> *d_inst = nullptr;
    BItem *d_seg = nullptr, *d_chunk = nullptr;
    long long *d_steps_left = nullptr;
    // unfinished members of the group being solved and their item prefix counts
    ActRec *d_act = nullptr;
    int *d_counts = nullptr;
    int *d_packed = nullptr;       // per table row: 1 if its sweeps go through the packed kernel
    size_t cap_inst = 0, cap_seg = 0, cap_chunk = 0, cap_act = 0, cap_packed = 0;
    // members with at least solo_items stencil items, and every member of a group of at most
    // kSoloAllMembers, sweep in their own launches (descriptor by value, as in the
    // single-instance step), concurrently on their own capture streams
    int solo_items = 0;
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    int ninst = 0;
    long long nseg_items = 0, nchunk_items = 0;
    std::vector<int> order;        // slot of each table row
    cudaGraphExec_t graph = nullptr;
    bool dirty = true;
    int nsm = 152, sweeps_per_check = 16, zseg = kZSeg;
    bool spc_auto = true;          // sweeps_per_check sized per group from its work at graph build
    // members are swept in groups whose working sets fit the L2 cache together; each group
    // has its own device-side convergence loop (0 = one group)
    size_t group_bytes = 0;
    struct Group {
        int inst0, inst1;         // table rows [inst0, inst1)
        long long seg0, nseg;     // range of its stencil items in d_seg
        std::vector<int> solo;    // rows swept in their own launches
        long long packed_items;   // items of the other rows (packed sweep launches)
        bool cheb;                // its members' solver: Chebyshev-accelerated (else damped Jacobi)
    };
    std::vector<Group> groups;
    std::vector<Ctl> last;         // per table row, after the last step
    std::vector<ep_step_stats> stats;
};

namespace {

ep_status bfail(ep_batch *b, ep_status st, const std::string &msg)
{
    if (b) b->err = msg;
    return st;
}

#define CKB(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            cudaGetLastError();                                                                     \
            return bfail(b, EP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
        }                                                                                           \
    } while (0)

// Rebuilds a handle's stencil work items with zseg planes per item (within
// the capacity allocated at set-up).
ep_status relayout_segments(ep_sim *s, int zseg)
{
    if (zseg == s->zseg) return EP_OK;
    std::vector<Seg> segs = build_segments(s->mask.data(), s->d.nx, s->d.ny, s->d.nz, zseg);
    if ((long long)segs.size() > s->max_items) return fail(s, EP_EINVAL, "segment capacity exceeded");
    CK(cudaMemcpyAsync(s->segs, segs.data(), sizeof(Seg) * segs.size(), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->nseg = (int)segs.size();
    s->zseg = zseg;
    if (s->sweep_graph) {
        cudaGraphExecDestroy(s->sweep_graph);
        s->sweep_graph = nullptr;
    }
    if (s->ie_graph) {
        cudaGraphExecDestroy(s->ie_graph);
        s->ie_graph = nullptr;
    }
    return EP_OK;
}

template <typename T>
ep_status grow(ep_batch *b, T **p, size_t *cap, size_t need)
{
    if (need <= *cap && *p) return EP_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    const size_t n = std::max<size_t>(need, 1);
    CKB(cudaMalloc((void **)p, sizeof(T) * n));
    *cap = n;
    return EP_OK;
}

ep_status rebuild_tables(ep_batch *b)
{
    b->order.clear();
    for (int i = 0; i < b->max_inst; ++i)
        if (b->slot[i]) b->order.push_back(i);
    // damped-Jacobi members first, then Chebyshev ones: a group holds one solver (its sweep instance)
    auto is_cheb = [&](int slot) {   // as Inst::solver: the Chebyshev solver with its interval known
        const ep_sim *m = b->slot[slot];
        return m->p.solver == EP_SOLVER_CHEBYSHEV && m->cheb_lmax > 0.0;
    };
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return !is_cheb(x) && is_cheb(y); });
    b->ninst = (int)b->order.size();
    std::vector<Inst<float>> insts;
    std::vector<BItem> segs, chunks;
    for (int r = 0; r < b->ninst; ++r) {
        ep_sim *s = b->slot[b->order[r]];
        insts.push_back(make_inst<float>(s));
        for (int i = 0; i < s->nchunk; ++i) chunks.push_back(BItem{r, i, s->nchunk, 0});
    }
    // groups of consecutive rows whose sweep working sets (iterate pair, right-hand side,
    // records: 20 bytes per grid voxel) together stay within group_bytes
    b->groups.clear();
    for (int r = 0; r < b->ninst;) {
        int r1 = r;
        size_t bytes = 0;
        const bool cheb = is_cheb(b->order[r]);
        do {
            bytes += 20 * (size_t)b->slot[b->order[r1]]->n;
            ++r1;
        } while (r1 < b->ninst && is_cheb(b->order[r1]) == cheb &&
                 (b->group_bytes == 0 || bytes + 20 * (size_t)b->slot[b->order[r1]]->n <= b->group_bytes));
        ep_batch::Group g;
        g.cheb = cheb;
        g.inst0 = r;
        g.inst1 = r1;
        g.seg0 = (long long)segs.size();
        std::vector<BItem> gs;
        for (int q = r; q < r1; ++q) {
            ep_sim *s = b->slot[b->order[q]];
            for (int i = 0; i < s->nseg; ++i) gs.push_back(BItem{q, i, s->nseg, 0});
        }
        // interleave the group's instances so that every part of the persistent grid sees
        // work of several instances (long instances do not end up on a few CTAs)
        std::stable_sort(gs.begin(), gs.end(), [](const BItem &x, const BItem &y) {
            return (x.item + 0.5) / x.nitems < (y.item + 0.5) / y.nitems;
        });
        segs.insert(segs.end(), gs.begin(), gs.end());
        g.nseg = (long long)gs.size();
        g.packed_items = 0;
        const bool few = r1 - r <= kSoloAllMembers;
        for (int q = r; q < r1; ++q) {
            ep_sim *s = b->slot[b->order[q]];
            if (few || s->nseg >= b->solo_items) g.solo.push_back(q);
            else g.packed_items += s->nseg;
        }
        b->groups.push_back(g);
        r = r1;
    }
    std::vector<int> packed(b->ninst, 1);
    for (const ep_batch::Group &g : b->groups)
        for (int q : g.solo) packed[q] = 0;
    b->nseg_items = (long long)segs.size();
    b->nchunk_items = (long long)chunks.size();
    ep_status st;
    if ((st = grow(b, &b->d_inst, &b->cap_inst, insts.size())) != EP_OK) return st;
    if ((st = grow(b, &b->d_seg, &b->cap_seg, segs.size())) != EP_OK) return st;
    if ((st = grow(b, &b->d_chunk, &b->cap_chunk, chunks.size())) != EP_OK) return st;
    if ((st = grow(b, &b->d_act, &b->cap_act, insts.size() + 1)) != EP_OK) return st;
    if ((st = grow(b, &b->d_packed, &b->cap_packed, insts.size())) != EP_OK) return st;
    if (!insts.empty()) {
        CKB(cudaMemcpyAsync(b->d_packed, packed.data(), sizeof(int) * packed.size(), cudaMemcpyHostToDevice,
                            b->stream));
        CKB(cudaMemcpyAsync(b->d_inst, insts.data(), sizeof(Inst<float>) * insts.size(), cudaMemcpyHostToDevice,
                            b->stream));
        CKB(cudaMemcpyAsync(b->d_seg, segs.data(), sizeof(BItem) * segs.size(), cudaMemcpyHostToDevice, b->stream));
        CKB(cudaMemcpyAsync(b->d_chunk, chunks.data(), sizeof(BItem) * chunks.size(), cudaMemcpyHostToDevice,
                            b->stream));
    }
    CKB(cudaStreamSynchronize(b->stream));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->last.assign(b->ninst, Ctl{});
    b->dirty = false;
    return EP_OK;
}

int grid_of(long long items, int cap) { return (int)std::max<long long>(1, std::min<long long>(items, cap)); }

// One graph runs a whole chunk of steps: an outer loop over the steps left
// (device counter) whose body is one step; inside it, the sweeps of all
// unfinished solves repeat until every member has converged (or hit its cap).
ep_status build_batch_graph(ep_batch *b)
{
    if (b->graph) return EP_OK;
    size_t need = 0;
    for (const ep_batch::Group &gr : b->groups) need = std::max(need, gr.solo.size());
    if (need && !b->ev_fork) CKB(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    while (b->aux.size() < need) {
        cudaStream_t a = nullptr;
        cudaEvent_t e = nullptr;
        CKB(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
        b->aux.push_back(a);
        CKB(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->ev_join.push_back(e);
    }
    cudaStream_t st = b->stream;
    const int gs = grid_of(b->nseg_items, 1 << 30);   // one CTA per stencil item
    const int gc = grid_of(b->nchunk_items, b->nsm * 4);
    const int ns = (int)b->nseg_items, nc = (int)b->nchunk_items;
    Inst<float> none;
    std::memset(&none, 0, sizeof(none));
    cudaGraph_t g = nullptr;
    CKB(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle ho = 0;
    CKB(cudaGraphConditionalHandleCreate(&ho, g, 1, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char po_buf[sizeof(cudaGraphNodeParams)] = {};
    cudaGraphNodeParams &po = *reinterpret_cast<cudaGraphNodeParams *>(po_buf);
    po.type = cudaGraphNodeTypeConditional;
    po.conditional.handle = ho;
    po.conditional.type = cudaGraphCondTypeWhile;
    po.conditional.size = 1;
    cudaGraphNode_t no;
    CKB(cudaGraphAddNode(&no, g, nullptr, nullptr, 0, &po));
    cudaGraph_t body = po.conditional.phGraph_out[0];
    // inner loop handles, one per group (bidomain only: a handle without its conditional
    // node is invalid); each is set to 1 before its loop starts
    const int ngroups = (int)b->groups.size();
    std::vector<cudaGraphConditionalHandle> hg(ngroups, 0);
    if (b->model == EP_BI)
        for (int gi = 0; gi < ngroups; ++gi) CKB(cudaGraphConditionalHandleCreate(&hg[gi], body, 1, 0));

    CKB(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (b->model == EP_MONO) k_stencil_batch<float, M_PAR_MONO><<<gs, kThreads, kSmemBytes<float, M_PAR_MONO>, st>>>(b->d_inst, b->d_seg);
    else k_stencil_batch<float, M_PAR_BI><<<gs, kThreads, kSmemBytes<float, M_PAR_BI>, st>>>(b->d_inst, b->d_seg);
    if (b->model == EP_BI) {
        k_stencil_batch<float, M_RHS><<<gs, kThreads, kSmemBytes<float, M_RHS>, st>>>(b->d_inst, b->d_seg);
        k_comp_mean_batch<float><<<gc, kRedThreads, 0, st>>>(b->d_inst, b->d_chunk, nc, (int)RED_B);
        k_comp_subtract_batch<float><<<gc, kRedThreads, 0, st>>>(b->d_inst, b->d_chunk, nc);
        for (int gi = 0; gi < ngroups; ++gi) {
            const ep_batch::Group &gr = b->groups[gi];
            const int gn = gr.inst1 - gr.inst0;
            const Inst<float> *gi_inst = b->d_inst + gr.inst0;
            const int *gi_packed = b->d_packed + gr.inst0;
            k_active_list<float><<<1, kActThreads, 0, st>>>(gi_inst, gi_packed, gn, b->d_act, b->d_counts, hg[gi]);
            // inner loop: sweeps of the unfinished members until every solve of the group is finished
            cudaStreamCaptureStatus cs;
            cudaGraph_t cg = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            const cudaGraphEdgeData *ed = nullptr;
            size_t nd = 0;
            CKB(cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, &ed, &nd));
            alignas(cudaGraphNodeParams) unsigned char pi_buf[sizeof(cudaGraphNodeParams)] = {};
            cudaGraphNodeParams &pi = *reinterpret_cast<cudaGraphNodeParams *>(pi_buf);
            pi.type = cudaGraphNodeTypeConditional;
            pi.conditional.handle = hg[gi];
            pi.conditional.type = cudaGraphCondTypeWhile;
            pi.conditional.size = 1;
            cudaGraphNode_t ni;
            CKB(cudaGraphAddNode(&ni, cg, deps, ed, nd, &pi));
            cudaGraph_t ibody = pi.conditional.phGraph_out[0];
            CKB(cudaStreamUpdateCaptureDependencies(st, &ni, nullptr, 1, cudaStreamSetCaptureDependencies));
            CKB(cudaStreamBeginCaptureToGraph(b->side, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            // solo members: their own sweep chains on forked streams (parallel graph branches)
            const int nsolo = (int)gr.solo.size();
            if (nsolo) CKB(cudaEventRecord(b->ev_fork, b->side));
            // sweeps between loop checks: about 1 ms of sweeps (a loop pass costs tens of us), or as set
            int spc = b->sweeps_per_check;
            if (b->spc_auto) {
                long long widest = gr.packed_items;
                for (int q : gr.solo) widest = std::max<long long>(widest, b->slot[b->order[q]]->nseg);
                const double waves = std::max(1.0, (double)widest / (double)(b->nsm * kMinBlocks));
                spc = (int)std::min(64.0, std::max(8.0, std::round(1000.0 / (15.0 * waves))));
            }
            for (int j = 0; j < nsolo; ++j) {
                cudaStream_t a = b->aux[j];
                CKB(cudaStreamWaitEvent(a, b->ev_fork, 0));
                const Inst<float> I = make_inst<float>(b->slot[b->order[gr.solo[j]]]);
                for (int i = 0; i < spc; ++i) {
                    if (gr.cheb) k_stencil<float, M_JAC_CHEB><<<I.nseg, kThreads, kSmemBytes<float, M_JAC_CHEB>, a>>>(I, no_io<float>());
                    else k_stencil<float, M_JAC><<<I.nseg, kThreads, kSmemBytes<float, M_JAC>, a>>>(I, no_io<float>());
                }
                CKB(cudaEventRecord(b->ev_join[j], a));
            }
            // the other members: packed sweeps over the unfinished ones
            if (gr.packed_items > 0)
                for (int i = 0; i < spc; ++i) {
                    const int gp = grid_of(gr.packed_items, 1 << 30);
                    if (gr.cheb) k_stencil_active<float, M_JAC_CHEB><<<gp, kThreads, kSmemBytes<float, M_JAC_CHEB>, b->side>>>(gi_inst, b->d_act, gn);
                    else k_stencil_active<float, M_JAC><<<gp, kThreads, kSmemBytes<float, M_JAC>, b->side>>>(gi_inst, b->d_act, gn);
                }
            for (int j = 0; j < nsolo; ++j) CKB(cudaStreamWaitEvent(b->side, b->ev_join[j], 0));
            k_active_list<float><<<1, kActThreads, 0, b->side>>>(gi_inst, gi_packed, gn, b->d_act, b->d_counts,
                                                                 hg[gi]);
            CKB(cudaStreamEndCapture(b->side, nullptr));
        }
        k_comp_mean_batch<float><<<gc, kRedThreads, 0, st>>>(b->d_inst, b->d_chunk, nc, (int)RED_X_FINAL);
        k_project_batch<float><<<gc, kRedThreads, 0, st>>>(b->d_inst, b->d_chunk, nc);
    }
    k_end_step<float><<<1, 256, 0, st>>>(b->d_inst, b->ninst, none);
    k_steps_cond<<<1, 1, 0, st>>>(b->d_steps_left, ho);
    CKB(cudaStreamEndCapture(st, nullptr));
    cudaGraphInstantiateParams ip;
    std::memset(&ip, 0, sizeof(ip));
    cudaError_t e = cudaGraphInstantiateWithParams(&b->graph, g, &ip);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        std::string why = std::string("batch graph instantiate: ") + cudaGetErrorString(e) +
                          " (result " + std::to_string((int)ip.result_out);
        if (ip.errNode_out) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(ip.errNode_out, &t) == cudaSuccess) why += ", node type " + std::to_string((int)t);
        }
        why += ")";
        if (const char *dump = std::getenv("EP_GRAPH_DOT")) cudaGraphDebugDotPrint(g, dump, cudaGraphDebugDotFlagsVerbose);
        cudaGetLastError();
        cudaGraphDestroy(g);
        return bfail(b, EP_ECUDA, why);
    }
    cudaGraphDestroy(g);
    return EP_OK;
}

}  // namespace

extern "C" {

ep_status ep_batch_create(int max_instances, size_t hbm_budget_bytes, void *cuda_stream, ep_batch **out)
{
    if (!out) return EP_EINVAL;
    *out = nullptr;
    if (max_instances < 1 || max_instances > 65536) return EP_EINVAL;
    ep_batch *b = new (std::nothrow) ep_batch();
    if (!b) return EP_ENOMEM;
    b->max_inst = max_instances;
    b->budget = hbm_budget_bytes;
    b->slot.assign(max_instances, nullptr);
    b->stats.assign(max_instances, ep_step_stats{});
    auto bad = [&](cudaError_t e) {
        cudaGetLastError();
        (void)e;
        if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
        if (b->side) cudaStreamDestroy(b->side);
        if (b->d_steps_left) cudaFree(b->d_steps_left);
        if (b->d_counts) cudaFree(b->d_counts);
        delete b;
        return EP_ECUDA;
    };
    cudaError_t e;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
        b->own_stream = true;
    }
    if ((e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return bad(e);
    if ((e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return bad(e);
    b->solo_items = b->nsm * kMinBlocks / 2;   // half a wave of resident sweep CTAs
    if ((e = cudaMalloc((void **)&b->d_steps_left, sizeof(long long))) != cudaSuccess) return bad(e);
    if ((e = cudaMalloc((void **)&b->d_counts, 2 * sizeof(int))) != cudaSuccess) return bad(e);
    *out = b;
    return EP_OK;
}

ep_status ep_batch_add(ep_batch *b, ep_sim *s, int *slot)
{
    if (!b || !s || !slot) return EP_EINVAL;
    if (s->d.precision != EP_FP32) return bfail(b, EP_EINVAL, "batched members must be FP32 handles");
    if (s->have_params && s->p.diffusion != EP_EXPLICIT)
        return bfail(b, EP_EINVAL, "implicit-diffusion handles are stepped by ep_step only");
    if (!s->torso.empty() || s->ecg_q[0] >= 0)
        return bfail(b, EP_EINVAL, "torso and ECG handles are stepped by ep_step only");
    if (s->have_params && s->p.solver == EP_SOLVER_GAUSS_SEIDEL)
        return bfail(b, EP_EINVAL, "Gauss-Seidel handles are stepped by ep_step only");
    if (b->model >= 0 && s->d.model != b->model)
        return bfail(b, EP_EINVAL, "batched members must share the model (monodomain or bidomain)");
    for (ep_sim *t : b->slot)
        if (t == s) return bfail(b, EP_EINVAL, "handle is already in the batch");
    int free_slot = -1;
    size_t used = 0;
    for (int i = 0; i < b->max_inst; ++i) {
        if (b->slot[i]) used += b->slot[i]->dev_bytes;
        else if (free_slot < 0) free_slot = i;
    }
    if (free_slot < 0) return bfail(b, EP_EBUSY, "batch is full");
    ep_status st = ensure_ready(s);
    if (st != EP_OK) return bfail(b, st, std::string("set-up of the handle failed: ") + s->err);
    if (b->budget && used + s->dev_bytes > b->budget)
        return bfail(b, EP_EREJECTED, "admission refused: device memory budget exceeded");
    if (s->stream) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return bfail(b, EP_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
    }
    st = relayout_segments(s, b->zseg);
    if (st != EP_OK) return bfail(b, st, s->err);
    b->slot[free_slot] = s;
    b->model = s->d.model;
    b->dirty = true;
    *slot = free_slot;
    return EP_OK;
}

ep_status ep_batch_remove(ep_batch *b, int slot)
{
    if (!b || slot < 0 || slot >= b->max_inst || !b->slot[slot]) return EP_EINVAL;
    b->slot[slot] = nullptr;
    b->dirty = true;
    bool any = false;
    for (ep_sim *t : b->slot) any = any || t;
    if (!any) b->model = -1;
    return EP_OK;
}

ep_status ep_batch_step(ep_batch *b, int n_steps)
{
    if (!b) return EP_EINVAL;
    if (n_steps < 0) return bfail(b, EP_EINVAL, "n_steps must be >= 0");
    ep_status st;
    if (b->dirty && (st = rebuild_tables(b)) != EP_OK) return st;
    if (b->ninst == 0 || n_steps == 0) return EP_OK;
    if ((st = build_batch_graph(b)) != EP_OK) return st;
    cudaStream_t s0 = b->stream;
    // members may have been stepped on their own streams before
    for (int r = 0; r < b->ninst; ++r) {
        ep_sim *s = b->slot[b->order[r]];
        CKB(cudaStreamSynchronize(s->stream));
        // flags of this call (non-finite, diverged, not converged) start clear
        const int zero[3] = {0, 0, 0};
        CKB(cudaMemcpyAsync((char *)s->ctl + offsetof(Ctl, nonfinite), zero, sizeof(zero), cudaMemcpyHostToDevice, s0));
    }
    const long long n = n_steps;
    CKB(cudaMemcpyAsync(b->d_steps_left, &n, sizeof(n), cudaMemcpyHostToDevice, s0));
    CKB(cudaGraphLaunch(b->graph, s0));
    for (int r = 0; r < b->ninst; ++r)
        CKB(cudaMemcpyAsync(&b->last[r], b->slot[b->order[r]]->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s0));
    CKB(cudaStreamSynchronize(s0));
    ep_status ret = EP_OK;
    for (int r = 0; r < b->ninst; ++r) {
        const int sl = b->order[r];
        ep_sim *s = b->slot[sl];
        const Ctl &c = b->last[r];
        s->step = c.step;
        ep_step_stats &x = b->stats[sl];
        x.iters = c.iters;
        x.rel_res = c.bnorm2 > 0.0 ? std::sqrt(c.rnorm2 / c.bnorm2) : 0.0;
        x.converged = !c.noconv;
        x.total_iters = c.total_iters;
        x.step = c.step;
        if (c.nonfinite) ret = EP_ENONFINITE;
        else if (c.noconv && ret == EP_OK) ret = EP_ENOCONV;
    }
    if (ret == EP_ENOCONV) b->err = "an elliptic solve reached max_iter or diverged";
    if (ret == EP_ENONFINITE) b->err = "non-finite value in a member's state";
    return ret;
}

ep_status ep_batch_slot_stats(ep_batch *b, int slot, ep_step_stats *stats)
{
    if (!b || !stats || slot < 0 || slot >= b->max_inst || !b->slot[slot]) return EP_EINVAL;
    *stats = b->stats[slot];
    return EP_OK;
}

ep_status ep_batch_autotune(ep_batch *b, int trial_sweeps)
{
    if (!b || trial_sweeps < 1) return EP_EINVAL;
    ep_status st;
    if (b->dirty && (st = rebuild_tables(b)) != EP_OK) return st;
    if (b->ninst == 0) return EP_OK;
    cudaStream_t s0 = b->stream;
    // snapshot the solve state of every member: v_e (x0) and the control block
    std::vector<void *> saved(b->ninst, nullptr);
    std::vector<Ctl> ctl0(b->ninst);
    auto release = [&]() {
        for (void *p : saved)
            if (p) cudaFree(p);
    };
    for (int r = 0; r < b->ninst; ++r) {
        ep_sim *s = b->slot[b->order[r]];
        CKB(cudaStreamSynchronize(s->stream));
        if (cudaMalloc(&saved[r], sizeof(float) * s->n) != cudaSuccess) {
            cudaGetLastError();
            release();
            return bfail(b, EP_ENOMEM, "autotune: no room for the state snapshot");
        }
        CKB(cudaMemcpyAsync(saved[r], s->x[0], sizeof(float) * s->n, cudaMemcpyDeviceToDevice, s0));
        CKB(cudaMemcpyAsync(&ctl0[r], s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s0));
    }
    CKB(cudaStreamSynchronize(s0));
    cudaEvent_t e0, e1;
    CKB(cudaEventCreate(&e0));
    CKB(cudaEventCreate(&e1));
    const int zsegs[3] = {8, 16, 32};
    const size_t gbytes[4] = {0, (size_t)192 << 20, (size_t)96 << 20, (size_t)48 << 20};
    double best = 1e300;
    int best_z = b->zseg;
    size_t best_g = b->group_bytes;
    for (int zi = 0; zi < 3 && st == EP_OK; ++zi) {
        for (int r = 0; r < b->ninst && st == EP_OK; ++r) st = relayout_segments(b->slot[b->order[r]], zsegs[zi]);
        if (st != EP_OK) break;
        for (int gi = 0; gi < 4 && st == EP_OK; ++gi) {
            b->group_bytes = gbytes[gi];
            if ((st = rebuild_tables(b)) != EP_OK) break;
            if (gi > 0 && b->groups.size() == 1) continue;   // same as one group
            // never-converging solves so that every trial sweep does its full work
            for (int r = 0; r < b->ninst; ++r) {
                Ctl c = ctl0[r];
                c.done = 0; c.sweep = 0; c.arrive = 0; c.jarrive = 0; c.thresh2 = -1.0; c.bnorm2 = 1e300;
                c.cycle0 = 0; c.r0n2 = 0.0;
                CKB(cudaMemcpyAsync(b->slot[b->order[r]]->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s0));
            }
            // one sweep of every group in turn, each group swept trial_sweeps times
            double ms_total = 0.0;
            for (const ep_batch::Group &gr : b->groups) {
                const int gs = grid_of(gr.nseg, 1 << 30);
                auto sweep = [&]() {
                    if (gr.cheb) k_stencil_batch<float, M_JAC_CHEB><<<gs, kThreads, kSmemBytes<float, M_JAC_CHEB>, s0>>>(b->d_inst, b->d_seg + gr.seg0);
                    else k_stencil_batch<float, M_JAC><<<gs, kThreads, kSmemBytes<float, M_JAC>, s0>>>(b->d_inst, b->d_seg + gr.seg0);
                };
                sweep();
                CKB(cudaEventRecord(e0, s0));
                for (int i = 0; i < trial_sweeps; ++i) sweep();
                CKB(cudaEventRecord(e1, s0));
                CKB(cudaEventSynchronize(e1));
                float ms = 0.f;
                CKB(cudaEventElapsedTime(&ms, e0, e1));
                ms_total += ms;
            }
            if (ms_total < best) {
                best = ms_total;
                best_z = zsegs[zi];
                best_g = gbytes[gi];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the members' solve state and apply the best layout
    for (int r = 0; r < b->ninst; ++r) {
        ep_sim *s = b->slot[b->order[r]];
        CKB(cudaMemcpyAsync(s->x[0], saved[r], sizeof(float) * s->n, cudaMemcpyDeviceToDevice, s0));
        CKB(cudaMemcpyAsync(s->ctl, &ctl0[r], sizeof(Ctl), cudaMemcpyHostToDevice, s0));
    }
    CKB(cudaStreamSynchronize(s0));
    release();
    if (st != EP_OK) return st;
    b->zseg = best_z;
    b->group_bytes = best_g;
    // sweeps between device loop checks: about 1 ms of sweeps, 8..64 (a loop pass costs tens of us)
    const double per_sweep_us = 1e3 * best / trial_sweeps;
    b->sweeps_per_check = (int)std::min(64.0, std::max(8.0, std::ceil(1000.0 / std::max(per_sweep_us, 1e-3))));
    b->spc_auto = false;
    for (int r = 0; r < b->ninst && st == EP_OK; ++r) st = relayout_segments(b->slot[b->order[r]], b->zseg);
    if (st != EP_OK) return st;
    return rebuild_tables(b);
}

ep_status ep_batch_set_schedule(ep_batch *b, int sweeps_per_check, int zseg, long long group_bytes)
{
    if (!b) return EP_EINVAL;
    if (sweeps_per_check < 0 || sweeps_per_check > 1024)
        return bfail(b, EP_EINVAL, "sweeps_per_check must be in [1, 1024] (0 keeps)");
    if (zseg != 0 && (zseg < kZSegMin || zseg > 256)) return bfail(b, EP_EINVAL, "zseg must be in [8, 256] (0 keeps)");
    if (sweeps_per_check) {
        b->sweeps_per_check = sweeps_per_check;
        b->spc_auto = false;
    }
    if (group_bytes >= 0) b->group_bytes = (size_t)group_bytes;
    if (zseg && zseg != b->zseg) {
        b->zseg = zseg;
        for (ep_sim *t : b->slot) {
            if (!t) continue;
            const ep_status st = relayout_segments(t, zseg);
            if (st != EP_OK) return bfail(b, st, t->err);
        }
    }
    b->dirty = true;
    return EP_OK;
}

ep_status ep_batch_get_info(ep_batch *b, ep_batch_info *info)
{
    if (!b || !info) return EP_EINVAL;
    ep_status st;
    if (b->dirty && (st = rebuild_tables(b)) != EP_OK) return st;
    info->instances = b->ninst;
    info->stencil_items = b->nseg_items;
    info->chunk_items = b->nchunk_items;
    size_t used = 0;
    for (ep_sim *s : b->slot)
        if (s) used += s->dev_bytes;
    info->device_bytes = used;
    info->budget_bytes = b->budget;
    info->sweeps_per_check = b->sweeps_per_check;
    info->zseg = b->zseg;
    info->group_bytes = b->group_bytes;
    info->groups = (int)b->groups.size();
    int solo = 0;
    for (const ep_batch::Group &g : b->groups) solo += (int)g.solo.size();
    info->solo_members = solo;
    return EP_OK;
}

const char *ep_batch_last_error(const ep_batch *b) { return b ? b->err.c_str() : "null batch"; }

void ep_batch_destroy(ep_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_seg) cudaFree(b->d_seg);
    if (b->d_chunk) cudaFree(b->d_chunk);
    if (b->d_act) cudaFree(b->d_act);
    if (b->d_packed) cudaFree(b->d_packed);
    for (cudaStream_t a : b->aux) cudaStreamDestroy(a);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->d_counts) cudaFree(b->d_counts);
    if (b->d_steps_left) cudaFree(b->d_steps_left);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

// ===========================================================================
// Served form: requests arrive over time and join a running batch
// (continuous batching).  One serving thread admits released requests in
// release order while a slot is free and the request's device footprint
// (set-up peak) fits the budget beside everything the server holds, sets them
// up, runs the batched step in chunks and retires each request when its steps
// are done.  Membership changes only between chunks; the batch rebuilds its
// tables and graph then.  Monodomain and bidomain requests go to separate
// batches, stepped one after the other in each chunk.
// ===========================================================================
namespace {

using SrvClock = std::chrono::steady_clock;

struct SrvReq {
    long long id = 0;
    ep_sim *sim = nullptr;
    int n_steps = 0, steps_done = 0, slot = -1, model = 0;
    int status = EP_OK, plan_status = EP_OK;
    bool cancel = false, busy = false, planned = false;
    double release = 0, t_admit = -1, t_done = -1;
    long long iters_base = 0, total_iters = 0;
    size_t peak = 0, bytes = 0;
};

}  // namespace

struct ep_server {
    ep_server_config cfg{};
    int device = 0;
    ep_batch *batch[2] = {nullptr, nullptr};   // by model
    std::thread thr, planner;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_plan;
    bool stop = false;
    bool blocked_on_results = false;   // nothing runs and the next request waits for memory held by results
    std::string err;
    SrvClock::time_point t0;
    std::deque<SrvReq *> queue;      // submitted, by release time then id
    std::vector<SrvReq *> active;    // batch members
    SrvReq *admitting = nullptr;     // being set up (between queue and active)
    std::deque<SrvReq *> finished;   // retired, not collected
    long long next_id = 1;
    size_t hbm_in_use = 0;           // bytes of held requests, plus the set-up reservation
    ep_server_stats st{};
    double now() const { return std::chrono::duration<double>(SrvClock::now() - t0).count(); }
};

namespace {

ep_status sfail(ep_server *v, ep_status st, const std::string &msg)
{
    v->err = msg;
    return st;
}

// Control block of a member after the batch's last step (nullptr if absent).
const Ctl *batch_member_ctl(const ep_batch *b, int slot)
{
    for (int r = 0; r < b->ninst && r < (int)b->last.size(); ++r)
        if (b->order[r] == slot) return &b->last[r];
    return nullptr;
}

// mu held.  A request leaves the server's queue or batch.
void srv_finish(ep_server *v, SrvReq *r, int status)
{
    if (status != EP_OK) r->status = status;
    r->t_done = v->now();
    v->finished.push_back(r);
    v->cv_done.notify_all();
}

void srv_erase(std::deque<SrvReq *> &q, SrvReq *r)
{
    auto it = std::find(q.begin(), q.end(), r);
    if (it != q.end()) q.erase(it);
}

void serve_loop(ep_server *v)
{
    cudaSetDevice(v->device);
    const size_t budget = v->cfg.hbm_budget_bytes;
    std::unique_lock<std::mutex> lk(v->mu);
    while (!v->stop) {
        // 1. cancelled members leave at this chunk boundary
        for (size_t i = 0; i < v->active.size();) {
            SrvReq *r = v->active[i];
            if (!r->cancel) {
                ++i;
                continue;
            }
            ep_batch_remove(v->batch[r->model], r->slot);
            v->active.erase(v->active.begin() + i);
            ++v->st.cancelled;
            srv_finish(v, r, EP_ECANCELLED);
        }
        // 2. admission of released requests, in release order
        while (!v->stop && !v->queue.empty() && v->queue.front()->release <= v->now() &&
               (int)v->active.size() < v->cfg.max_slots) {
            SrvReq *r = v->queue.front();
            if (!r->planned) break;   // the planner thread is on it; chunks go on meanwhile
            if (r->plan_status != EP_OK) {
                srv_erase(v->queue, r);
                srv_finish(v, r, r->plan_status);
                continue;
            }
            if (budget && r->peak > budget) {
                srv_erase(v->queue, r);
                ++v->st.rejected;
                srv_finish(v, r, EP_EREJECTED);
                continue;
            }
            if (r->cancel) {
                srv_erase(v->queue, r);
                ++v->st.cancelled;
                srv_finish(v, r, EP_ECANCELLED);
                continue;
            }
            if (v->cfg.max_active_items > 0 && !v->active.empty()) {   // enough work on the device already
                long long items = r->sim->nseg;
                for (const SrvReq *q : v->active) items += q->sim->nseg;
                if (items > v->cfg.max_active_items) break;
            }
            if (budget && v->hbm_in_use + r->peak > budget) {   // wait for memory to be released
                if (v->active.empty() && !v->finished.empty() && !v->blocked_on_results) {
                    v->blocked_on_results = true;
                    v->cv_done.notify_all();
                }
                break;
            }
            v->blocked_on_results = false;
            srv_erase(v->queue, r);
            v->admitting = r;
            v->hbm_in_use += r->peak;
            v->st.hbm_peak = std::max(v->st.hbm_peak, v->hbm_in_use);
            lk.unlock();
            ep_status as = ensure_ready(r->sim);
            int slot = -1;
            Ctl c0;
            std::memset(&c0, 0, sizeof(c0));
            if (as == EP_OK) as = ep_batch_add(v->batch[r->model], r->sim, &slot);
            if (as == EP_OK) {
                if (cudaMemcpyAsync(&c0, r->sim->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, r->sim->stream) != cudaSuccess ||
                    cudaStreamSynchronize(r->sim->stream) != cudaSuccess) {
                    cudaGetLastError();
                    as = EP_ECUDA;
                }
            }
            lk.lock();
            v->admitting = nullptr;
            v->hbm_in_use -= r->peak;
            r->bytes = r->sim->dev_bytes;
            v->hbm_in_use += r->bytes;
            if (as != EP_OK) {
                if (slot >= 0) ep_batch_remove(v->batch[r->model], slot);
                v->err = std::string("admission of request ") + std::to_string(r->id) + " failed: " + r->sim->err +
                         " " + ep_batch_last_error(v->batch[r->model]);
                srv_finish(v, r, as);
                continue;
            }
            r->slot = slot;
            r->iters_base = c0.total_iters;
            r->t_admit = v->now();
            v->active.push_back(r);
            ++v->st.admitted;
        }
        if (v->stop) break;
        // 3. nothing to run: sleep until the next release, a submission, a collect or a cancel
        if (v->active.empty()) {
            if (v->queue.empty()) {
                v->cv_work.wait(lk);
            } else {
                const double wait = v->queue.front()->release - v->now();
                if (wait > 0) v->cv_work.wait_for(lk, std::chrono::duration<double>(std::min(wait, 3600.0)));
                else v->cv_work.wait_for(lk, std::chrono::milliseconds(100));   // blocked on memory held by results
            }
            continue;
        }
        // 4. one chunk: at most chunk_steps, and no member passes its step count
        int k[2] = {v->cfg.chunk_steps, v->cfg.chunk_steps};
        bool has[2] = {false, false};
        for (SrvReq *r : v->active) {
            k[r->model] = std::min(k[r->model], r->n_steps - r->steps_done);
            has[r->model] = true;
        }
        lk.unlock();
        const double tb = v->now();
        ep_status bs[2] = {EP_OK, EP_OK};
        for (int m = 0; m < 2; ++m)
            if (has[m]) bs[m] = ep_batch_step(v->batch[m], k[m]);
        const double te = v->now();
        lk.lock();
        v->st.busy_s += te - tb;
        ++v->st.chunks;
        long long vs = 0;
        for (size_t i = 0; i < v->active.size();) {
            SrvReq *r = v->active[i];
            const ep_status b = bs[r->model];
            int stat = EP_OK;
            if (b == EP_OK || b == EP_ENOCONV || b == EP_ENONFINITE) {
                r->steps_done += k[r->model];
                vs += (long long)k[r->model] * r->sim->n_tissue;
                if (const Ctl *c = batch_member_ctl(v->batch[r->model], r->slot)) {
                    r->total_iters = c->total_iters - r->iters_base;
                    if (c->nonfinite) stat = EP_ENONFINITE;
                    else if (c->noconv) r->status = EP_ENOCONV;   // kept: the request still runs to its end
                }
            } else {   // the batched launch failed: its members fail with it
                stat = b;
                v->err = std::string("batched step failed: ") + ep_batch_last_error(v->batch[r->model]);
            }
            if (stat != EP_OK || r->steps_done >= r->n_steps) {
                ep_batch_remove(v->batch[r->model], r->slot);
                r->slot = -1;
                v->active.erase(v->active.begin() + i);
                ++v->st.completed;
                srv_finish(v, r, stat);
                continue;
            }
            ++i;
        }
        v->st.voxel_steps += vs;
    }
}

// Host planning of released requests (mask analysis and exact footprint),
// ahead of admission and while the GPU runs chunks.
void plan_loop(ep_server *v)
{
    std::unique_lock<std::mutex> lk(v->mu);
    while (!v->stop) {
        SrvReq *r = nullptr;
        double next = -1.0;   // release time of the next unplanned request, if not yet released
        for (SrvReq *q : v->queue) {
            if (q->planned || q->busy) continue;
            if (q->release <= v->now()) r = q;
            else next = q->release;
            break;
        }
        if (!r) {
            if (next >= 0.0) v->cv_plan.wait_for(lk, std::chrono::duration<double>(std::min(next - v->now(), 3600.0)));
            else v->cv_plan.wait(lk);
            continue;
        }
        r->busy = true;
        lk.unlock();
        const ep_status ps = plan_layout(r->sim);
        lk.lock();
        r->busy = false;
        r->planned = true;
        r->plan_status = ps;
        r->peak = r->sim->ready ? r->sim->dev_bytes : r->sim->fp_peak;
        v->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

ep_status ep_server_create(const ep_server_config *cfg, ep_server **out)
{
    if (!out) return EP_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->max_slots < 1 || cfg->max_slots > 65536 || cfg->chunk_steps < 1 || cfg->sweeps_per_check < 0 ||
        cfg->sweeps_per_check > 1024 || cfg->max_active_items < 0)
        return EP_EINVAL;
    ep_server *v = new (std::nothrow) ep_server();
    if (!v) return EP_ENOMEM;
    v->cfg = *cfg;
    v->t0 = SrvClock::now();
    cudaError_t e = cudaGetDevice(&v->device);
    ep_status st = e == cudaSuccess ? EP_OK : EP_ECUDA;
    for (int m = 0; m < 2 && st == EP_OK; ++m) {
        st = ep_batch_create(cfg->max_slots, 0, cfg->cuda_stream, &v->batch[m]);
        if (st == EP_OK && cfg->sweeps_per_check) st = ep_batch_set_schedule(v->batch[m], cfg->sweeps_per_check, 0, -1);
    }
    if (st != EP_OK) {
        cudaGetLastError();
        for (ep_batch *b : v->batch) ep_batch_destroy(b);
        delete v;
        return st;
    }
    try {
        v->planner = std::thread(plan_loop, v);
        v->thr = std::thread(serve_loop, v);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(v->mu);
            v->stop = true;
        }
        v->cv_plan.notify_all();
        if (v->planner.joinable()) v->planner.join();
        for (ep_batch *b : v->batch) ep_batch_destroy(b);
        delete v;
        return EP_ENOMEM;
    }
    *out = v;
    return EP_OK;
}

ep_status ep_server_submit(ep_server *v, ep_sim *sim, int n_steps, double release_s, long long *id)
{
    if (!v || !sim || !id || n_steps < 1) return EP_EINVAL;
    if (sim->d.precision != EP_FP32) return sfail(v, EP_EINVAL, "served requests must be FP32 handles");
    if (sim->have_params && sim->p.diffusion != EP_EXPLICIT)
        return sfail(v, EP_EINVAL, "implicit-diffusion handles are stepped by ep_step only");
    if (!sim->torso.empty() || sim->ecg_q[0] >= 0)
        return sfail(v, EP_EINVAL, "torso and ECG handles are stepped by ep_step only");
    if (!sim->have_mask || !sim->have_params) return sfail(v, EP_ESTATE, "a request needs its mask and parameters set");
    std::lock_guard<std::mutex> lk(v->mu);
    if (v->stop) return sfail(v, EP_ESTATE, "server is shutting down");
    auto holds = [&](const SrvReq *r) { return r && r->sim == sim; };
    if (std::any_of(v->queue.begin(), v->queue.end(), holds) || std::any_of(v->active.begin(), v->active.end(), holds) ||
        std::any_of(v->finished.begin(), v->finished.end(), holds) || holds(v->admitting))
        return sfail(v, EP_EINVAL, "handle is already held by the server");
    SrvReq *r = new (std::nothrow) SrvReq();
    if (!r) return EP_ENOMEM;
    r->id = v->next_id++;
    r->sim = sim;
    r->n_steps = n_steps;
    r->model = sim->d.model == EP_BI ? 1 : 0;
    r->release = std::max(release_s, v->now());
    auto pos = std::upper_bound(v->queue.begin(), v->queue.end(), r->release,
                                [](double t, const SrvReq *q) { return t < q->release; });
    v->queue.insert(pos, r);
    ++v->st.submitted;
    *id = r->id;
    v->cv_work.notify_all();
    v->cv_plan.notify_all();
    return EP_OK;
}

ep_status ep_server_cancel(ep_server *v, long long id)
{
    if (!v) return EP_EINVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    for (SrvReq *r : v->queue) {
        if (r->id != id) continue;
        if (r->busy) {
            r->cancel = true;
        } else {
            srv_erase(v->queue, r);
            ++v->st.cancelled;
            srv_finish(v, r, EP_ECANCELLED);
        }
        v->cv_work.notify_all();
        return EP_OK;
    }
    for (SrvReq *r : v->active)
        if (r->id == id) {
            r->cancel = true;
            return EP_OK;
        }
    if (v->admitting && v->admitting->id == id) {
        v->admitting->cancel = true;
        return EP_OK;
    }
    return sfail(v, EP_EINVAL, "no queued or running request with this id");
}

ep_status ep_server_collect(ep_server *v, ep_request_result *out, int max_results, int *n_out, double wait_s)
{
    if (!v || !out || max_results < 1 || !n_out) return EP_EINVAL;
    *n_out = 0;
    std::unique_lock<std::mutex> lk(v->mu);
    if (v->finished.empty() && wait_s > 0)
        v->cv_done.wait_for(lk, std::chrono::duration<double>(std::min(wait_s, 1e6)),
                            [&] { return !v->finished.empty() || v->stop; });
    int n = 0;
    if (!v->finished.empty()) v->blocked_on_results = false;
    while (n < max_results && !v->finished.empty()) {
        SrvReq *r = v->finished.front();
        v->finished.pop_front();
        ep_request_result &o = out[n++];
        o.id = r->id;
        o.status = r->status;
        o.steps_done = r->steps_done;
        o.n_tissue = r->sim->n_tissue;
        o.total_iters = r->total_iters;
        o.t_release_s = r->release;
        o.t_admit_s = r->t_admit;
        o.t_done_s = r->t_done;
        o.device_bytes = r->bytes;
        o.sim = r->sim;
        v->hbm_in_use -= r->bytes;
        delete r;
    }
    *n_out = n;
    if (n) v->cv_work.notify_all();
    return EP_OK;
}

ep_status ep_server_drain(ep_server *v, double timeout_s)
{
    if (!v) return EP_EINVAL;
    std::unique_lock<std::mutex> lk(v->mu);
    auto idle = [&] { return (v->queue.empty() && v->active.empty() && !v->admitting) || v->stop; };
    auto stuck = [&] { return v->blocked_on_results && v->active.empty() && !v->admitting; };
    auto done = [&] { return idle() || stuck(); };
    if (timeout_s < 0) v->cv_done.wait(lk, done);
    else if (!v->cv_done.wait_for(lk, std::chrono::duration<double>(std::min(timeout_s, 1e6)), done))
        return sfail(v, EP_EBUSY, "requests still pending at the timeout");
    if (!idle()) return sfail(v, EP_EBUSY, "admission waits for device memory held by uncollected results");
    return EP_OK;
}

ep_status ep_server_get_stats(ep_server *v, ep_server_stats *out)
{
    if (!v || !out) return EP_EINVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    *out = v->st;
    out->queued = (int)v->queue.size();
    out->active = (int)v->active.size() + (v->admitting ? 1 : 0);
    out->finished = (int)v->finished.size();
    out->hbm_in_use = v->hbm_in_use;
    out->now_s = v->now();
    return EP_OK;
}

double ep_server_now(const ep_server *v)
{
    return v ? v->now() : 0.0;
}

const char *ep_server_last_error(const ep_server *v) { return v ? v->err.c_str() : "null server"; }

void ep_server_destroy(ep_server *v)
{
    if (!v) return;
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stop = true;
    }
    v->cv_work.notify_all();
    v->cv_done.notify_all();
    v->cv_plan.notify_all();
    if (v->thr.joinable()) v->thr.join();
    if (v->planner.joinable()) v->planner.join();
    for (SrvReq *r : v->active) {
        ep_batch_remove(v->batch[r->model], r->slot);
        ep_destroy(r->sim);
        delete r;
    }
    for (auto *q : {&v->queue, &v->finished})
        for (SrvReq *r : *q) {
            ep_destroy(r->sim);
            delete r;
        }
    for (ep_batch *b : v->batch) ep_batch_destroy(b);
    delete v;
}

}  // extern "C"
