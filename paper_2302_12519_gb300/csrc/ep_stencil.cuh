// ep_stencil.cuh -- the z-marching stencil kernels of the voxel electrophysiology step.
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
// Work decomposition (GB300 design; the paper runs one thread per matrix row):
// a CTA owns 30 x kTileY output voxels of the x-y plane and marches through a
// z-range.  Warp w holds voxel rows (y0 + w - 1, y0 + w); lane l holds voxel
// column x0 - 1 + l, so x-neighbours come from warp shuffles.  Each warp forms
// the vertex row between its two voxel rows; the vertex row below comes from
// warp w - 1 through shared memory (one barrier per z-plane).  Tissue flags
// are 0/1 multipliers, so masking costs one multiply; the fibre outer
// products of a column are summed once and the left column's sum arrives by
// shuffle.  The plane loop is unrolled by two with two state records that
// swap roles, so nothing is copied between planes, and the loads of plane
// k + 1 are issued before plane k is processed.  The conductivity sums are
// rebuilt from the fp32 fibre records on every pass: on this GPU recomputing
// them costs less than streaming precomputed per-vertex FP32 coefficients
// (24 bytes a vertex; measured 67.7 against 72.4 us a sweep on the 256^3
// biventricular workload, the coefficient tiles brought in by TMA).
//
// The same item body serves the single-instance kernels (descriptor passed by
// value) and the batched persistent kernels (descriptor read from a device
// table, items of all instances packed in one list).
//
// With a conducting torso (M_JAC_BATH, M_APPLY_BATH) the records cover tissue
// + torso, torso voxels tagged, and every vertex carries two terms: the one
// above over tissue pairs, and Fo_a = ro_a^2 sig_o nB go_a over the pairs of
// any two domain voxels (go_a their summed differences, ro_a = 1 / their
// count, nB the torso voxels of the block).  Each term is scattered with its
// own pair flags.
#pragma once

#include "ep_common.cuh"

namespace gbep {

template <typename real>
__device__ __forceinline__ real rcp_count(real n)
{
    return n > real(0.5) ? real(1) / n : real(0);
}
template <>
__device__ __forceinline__ float rcp_count<float>(float n)
{
    return n > 0.5f ? __fdividef(1.0f, n) : 0.0f;   // n in {1, 2, 3, 4}
}

// Operand of M_APPLY (out = L_{sL,sT} u) and M_APPLY_BATH (the same plus the
// torso term of the descriptor's sig_o).
template <typename real>
struct ApplyIO {
    const real *u;
    real *out;
    real sT, dS;
};

// Per-item constants and pointers, resolved once at the start of an item.
template <typename real>
struct Op {
    const float4 *rec;
    const real *src, *w, *ve, *b;   // loads
    const real *inv;                // implicit sweep: 1 / (1 + a D_i)
    real *out, *wout, *tact;        // stores (PAR: v, w, t_act; RHS: b; APPLY: out; JAC, IE: next iterate;
    real *out2;                     //         IE_RHS: f, w, and v* in out2)
    real sT, dS, C, coef;
    real so;           // torso conductivity of the torso term (two-term modes)
    double tn, dt_d;
    int nz;
    int cheb;          // Jacobi sweep accelerated by the Chebyshev semi-iteration
    real cheb_w;       // its weight for this sweep
    // correction form, bits: kRestart = first sweep of a cycle (e starts from 0: the output
    // is coef D^-1 r, and r becomes the cycle's right-hand side, stored over b); kFold = add
    // the iterate read (the old cycle's e) into x0; kPrev0 = the cycle's previous iterate is 0
    // (Chebyshev)
    int cform;
    int colour;        // eight-colour sweep: the colour this launch updates
};

constexpr int kRestart = 1, kFold = 2, kPrev0 = 4;

// Loads of one plane for a lane's two voxel rows (lo = y0 + w - 1, hi = y0 + w).
template <typename real, int MODE>
struct Ld {
    float4 rLo, rHi;   // fp32 records
    real uLo, uHi;
    real wLo, wHi;     // PAR
    real veLo, veHi;   // PAR_BI
    real bLo;          // JAC: b; IE: f
    real iLo;          // IE: 1 / (1 + a D_i); JAC with the Chebyshev solver: x_{k-1} of row lo
};

// What the next plane needs from this one.
template <typename real>
struct St {
    real uLo, uHi, uLoL, uHiL;   // values of own / left column (0 off the tissue)
    real tLo, tHi, tLoL, tHiL;   // tissue 0/1
    real nT;                     // tissue count of the four voxels of this plane
    real Y[6];                   // sum of f f^T over the four voxels of this plane
    real sx, cx;                 // masked x-differences of this plane and their count
    real sy, cy;                 // masked y-differences of this plane and their count
    real FB[3], FA[3];           // vertex fluxes of the vertex plane below: own row, row below
    real tYm;                    // tissue of voxel (x, lo - 1) in this plane
    real tzm;                    // tissue of voxel (x, lo) in the plane below
    real e0, e1, e2;             // output voxel (x, lo): JAC b, 1/Dhat ; PAR v*, w+, v
    // torso term (two-term modes): the same over domain voxels (tissue or torso)
    real dLo, dHi, dLoL, dHiL;   // domain 0/1
    real nB;                     // torso voxels of the four voxels of this plane
    real sxd, cxd, syd, cyd;     // masked differences over domain pairs and their counts
    real FBo[3], FAo[3];         // torso-term vertex fluxes
    real dYm, dzm;               // domain flags of (x, lo - 1) here and of (x, lo) below
};

// Vertex-flux exchange of the torso term between warps (the row's tissue and
// domain flags travel together in sT as t + d).
template <typename real>
struct TorsoSmem {
    real sFo[2][3][kWarps][32];
};

template <typename real, int MODE>
__device__ __forceinline__ void load_plane(const Op<real> &o, int k, bool lo_in, bool hi_in, int qlo, int qhi,
                                           int plane, Ld<real, MODE> &L)
{
    const bool kin = (unsigned)k < (unsigned)o.nz;
    L.rLo = L.rHi = make_float4(0.f, 0.f, 0.f, kNonTissueW);
    L.uLo = L.uHi = L.veLo = L.veHi = L.bLo = L.iLo = real(0);
    L.wLo = L.wHi = real(1);
    if (kin && lo_in) {
        const int q = qlo + k * plane;
        L.rLo = __ldg(o.rec + q);
        L.uLo = __ldg(o.src + q);
        if (MODE == M_PAR_MONO || MODE == M_PAR_BI || MODE == M_IE_RHS) L.wLo = __ldg(o.w + q);
        if (MODE == M_PAR_BI || MODE == M_IE_RHS) L.veLo = __ldg(o.ve + q);
        if (kJac<MODE>) L.bLo = __ldg(o.b + q);
        if (kCheb<MODE> && o.cheb) L.iLo = o.out[q];   // x_{k-1}: this thread overwrites it one plane later
    }
    if (kin && hi_in) {
        const int q = qhi + k * plane;
        L.rHi = __ldg(o.rec + q);
        L.uHi = __ldg(o.src + q);
        if (MODE == M_PAR_MONO || MODE == M_PAR_BI || MODE == M_IE_RHS) L.wHi = __ldg(o.w + q);
        if (MODE == M_PAR_BI || MODE == M_IE_RHS) L.veHi = __ldg(o.ve + q);
    }
}

struct Lane {
    int lane, wid, x, ylo;
    int qlo, plane;
    bool out_lane;
};

// Process plane k: P = state of plane k - 1, C receives the state of plane k.
// Forms the vertex row between rows lo/hi at vertex plane k (k > kbeg) and
// writes voxel (x, lo, k - 1) (k > kbeg + 1).
template <typename real, int MODE>
__device__ __forceinline__ void plane_step(const Inst<real> &I, const Op<real> &o, const Lane &g, int k,
                                           bool do_vertex, bool do_output, const St<real> &P, St<real> &C,
                                           const Ld<real, MODE> &L, real (*sF)[3][kWarps][32],
                                           real (*sT)[kWarps][32], TorsoSmem<real> *ts, bool check, float &acc)
{
    constexpr bool TT = kTwoTerm<MODE>;
    // ---- decode the two voxels of the lane ----
    const bool dlo = rec_tissue(L.rLo), dhi = rec_tissue(L.rHi);   // in the records' domain
    const bool tlo = TT ? dlo && !rec_bath(L.rLo) : dlo;           // tissue
    const bool thi = TT ? dhi && !rec_bath(L.rHi) : dhi;
    const real flo0 = (real)L.rLo.x, flo1 = (real)L.rLo.y, flo2 = (real)L.rLo.z;
    const real fhi0 = (real)L.rHi.x, fhi1 = (real)L.rHi.y, fhi2 = (real)L.rHi.z;
    real ulo, uhi;
    C.e0 = C.e1 = C.e2 = real(0);
    if (MODE == M_PAR_MONO || MODE == M_PAR_BI || MODE == M_IE_RHS) {
        real vs, wn, vs2, wn2;
        ms_step(I, o.tn, L.uLo, L.wLo, g.x, g.ylo, k, vs, wn);
        ms_step(I, o.tn, L.uHi, L.wHi, g.x, g.ylo + 1, k, vs2, wn2);
        if (MODE == M_IE_RHS) {   // the stencil acts on ve alone
            ulo = tlo ? L.veLo : real(0);
            uhi = thi ? L.veHi : real(0);
        } else {
            ulo = tlo ? ((MODE == M_PAR_BI) ? vs + L.veLo : vs) : real(0);
            uhi = thi ? ((MODE == M_PAR_BI) ? vs2 + L.veHi : vs2) : real(0);
        }
        C.e0 = vs; C.e1 = wn; C.e2 = L.uLo;
    } else {
        ulo = dlo ? L.uLo : real(0);
        uhi = dhi ? L.uHi : real(0);
        if (kJac<MODE>) { C.e0 = L.bLo; C.e1 = (real)L.rLo.w; C.e2 = L.iLo; }
        if (MODE == M_IE) { C.e0 = L.bLo; C.e1 = L.iLo; }
    }
    C.uLo = ulo;
    C.uHi = uhi;
    C.tLo = tlo ? real(1) : real(0);
    C.tHi = thi ? real(1) : real(0);
    C.uLoL = __shfl_up_sync(kFull, ulo, 1);
    C.uHiL = __shfl_up_sync(kFull, uhi, 1);
    C.tLoL = __shfl_up_sync(kFull, C.tLo, 1);
    C.tHiL = __shfl_up_sync(kFull, C.tHi, 1);
    C.tzm = P.tLo;
    // outer products of the lane's column (fibres are zero off the tissue), then add the left column
    real Zo[6];
    Zo[0] = flo0 * flo0 + fhi0 * fhi0;
    Zo[1] = flo1 * flo1 + fhi1 * fhi1;
    Zo[2] = flo2 * flo2 + fhi2 * fhi2;
    Zo[3] = flo0 * flo1 + fhi0 * fhi1;
    Zo[4] = flo0 * flo2 + fhi0 * fhi2;
    Zo[5] = flo1 * flo2 + fhi1 * fhi2;
#pragma unroll
    for (int j = 0; j < 6; ++j) C.Y[j] = Zo[j] + __shfl_up_sync(kFull, Zo[j], 1);
    C.nT = (C.tLo + C.tHi) + (C.tLoL + C.tHiL);
    // pair differences of this plane: x (left -> own) in rows lo/hi, y (lo -> hi) in columns own/left
    const real cxlo = C.tLo * C.tLoL, cxhi = C.tHi * C.tHiL;
    C.sx = cxlo * (ulo - C.uLoL) + cxhi * (uhi - C.uHiL);
    C.cx = cxlo + cxhi;
    const real cyo = C.tLo * C.tHi, cyl = C.tLoL * C.tHiL;
    C.sy = cyo * (uhi - ulo) + cyl * (C.uHiL - C.uLoL);
    C.cy = cyo + cyl;
    if constexpr (TT) {   // the same over domain pairs
        C.dLo = dlo ? real(1) : real(0);
        C.dHi = dhi ? real(1) : real(0);
        C.dLoL = __shfl_up_sync(kFull, C.dLo, 1);
        C.dHiL = __shfl_up_sync(kFull, C.dHi, 1);
        C.dzm = P.dLo;
        C.nB = ((C.dLo + C.dHi) + (C.dLoL + C.dHiL)) - C.nT;
        const real dxlo = C.dLo * C.dLoL, dxhi = C.dHi * C.dHiL;
        C.sxd = dxlo * (ulo - C.uLoL) + dxhi * (uhi - C.uHiL);
        C.cxd = dxlo + dxhi;
        const real dyo = C.dLo * C.dHi, dyl = C.dLoL * C.dHiL;
        C.syd = dyo * (uhi - ulo) + dyl * (C.uHiL - C.uLoL);
        C.cyd = dyo + dyl;
    }

    // ---- vertex (x - 1/2, lo + 1/2, k - 1/2) ----
    real F0 = real(0), F1 = real(0), F2 = real(0);
    if (do_vertex) {
        const real czlo = P.tLo * C.tLo, czhi = P.tHi * C.tHi, czlol = P.tLoL * C.tLoL, czhil = P.tHiL * C.tHiL;
        const real gz = czlo * (ulo - P.uLo) + czhi * (uhi - P.uHi) + czlol * (C.uLoL - P.uLoL) +
                        czhil * (C.uHiL - P.uHiL);
        const real nz = (czlo + czhi) + (czlol + czhil);
        const real gx = P.sx + C.sx, nx = P.cx + C.cx;
        const real gy = P.sy + C.sy, ny = P.cy + C.cy;
        const real rx = rcp_count(nx), ry = rcp_count(ny), rz = rcp_count(nz);
        const real hx = gx * rx, hy = gy * ry, hz = gz * rz;
        const real iso = o.sT * (P.nT + C.nT);
        const real M0 = P.Y[0] + C.Y[0], M1 = P.Y[1] + C.Y[1], M2 = P.Y[2] + C.Y[2];
        const real M3 = P.Y[3] + C.Y[3], M4 = P.Y[4] + C.Y[4], M5 = P.Y[5] + C.Y[5];
        F0 = rx * (iso * hx + o.dS * (M0 * hx + M3 * hy + M4 * hz));
        F1 = ry * (iso * hy + o.dS * (M3 * hx + M1 * hy + M5 * hz));
        F2 = rz * (iso * hz + o.dS * (M4 * hx + M5 * hy + M2 * hz));
    }
    real Fo0 = real(0), Fo1 = real(0), Fo2 = real(0);
    if constexpr (TT) {
        if (do_vertex) {
            const real dzlo = P.dLo * C.dLo, dzhi = P.dHi * C.dHi, dzlol = P.dLoL * C.dLoL, dzhil = P.dHiL * C.dHiL;
            const real gzd = dzlo * (ulo - P.uLo) + dzhi * (uhi - P.uHi) + dzlol * (C.uLoL - P.uLoL) +
                             dzhil * (C.uHiL - P.uHiL);
            const real rxd = rcp_count(P.cxd + C.cxd), ryd = rcp_count(P.cyd + C.cyd),
                       rzd = rcp_count((dzlo + dzhi) + (dzlol + dzhil));
            const real ko = o.so * (P.nB + C.nB);
            Fo0 = rxd * rxd * ko * (P.sxd + C.sxd);
            Fo1 = ryd * ryd * ko * (P.syd + C.syd);
            Fo2 = rzd * rzd * ko * gzd;
        }
    }
    // ---- exchange vertex rows between warps (buffer by plane parity) ----
    const int par = k & 1;
    sF[par][0][g.wid][g.lane] = F0;
    sF[par][1][g.wid][g.lane] = F1;
    sF[par][2][g.wid][g.lane] = F2;
    sT[par][g.wid][g.lane] = TT ? C.tLo + C.dLo : C.tLo;
    if constexpr (TT) {
        ts->sFo[par][0][g.wid][g.lane] = Fo0;
        ts->sFo[par][1][g.wid][g.lane] = Fo1;
        ts->sFo[par][2][g.wid][g.lane] = Fo2;
    }
    __syncthreads();
    C.FB[0] = F0; C.FB[1] = F1; C.FB[2] = F2;
    if (g.wid >= 1) {
        C.FA[0] = sF[par][0][g.wid - 1][g.lane];
        C.FA[1] = sF[par][1][g.wid - 1][g.lane];
        C.FA[2] = sF[par][2][g.wid - 1][g.lane];
        C.tYm = sT[par][g.wid - 1][g.lane];
        if constexpr (TT) {   // unpack t + d (t <= d)
            C.dYm = C.tYm > real(0.5) ? real(1) : real(0);
            C.tYm = C.tYm > real(1.5) ? real(1) : real(0);
        }
    } else {
        C.FA[0] = C.FA[1] = C.FA[2] = C.tYm = real(0);
    }
    if constexpr (TT) {
        C.FBo[0] = Fo0; C.FBo[1] = Fo1; C.FBo[2] = Fo2;
        if (g.wid >= 1) {
            C.FAo[0] = ts->sFo[par][0][g.wid - 1][g.lane];
            C.FAo[1] = ts->sFo[par][1][g.wid - 1][g.lane];
            C.FAo[2] = ts->sFo[par][2][g.wid - 1][g.lane];
        } else {
            C.FAo[0] = C.FAo[1] = C.FAo[2] = C.dYm = real(0);
        }
    }

    // ---- output voxel (x, lo, k - 1) ----
    if (do_output) {
        const real phxm = (P.FA[0] + C.FA[0]) + (P.FB[0] + C.FB[0]);
        const real phxp = __shfl_down_sync(kFull, phxm, 1);
        const real psyA = P.FA[1] + C.FA[1], psyB = P.FB[1] + C.FB[1];
        const real phym = psyA + __shfl_down_sync(kFull, psyA, 1);
        const real phyp = psyB + __shfl_down_sync(kFull, psyB, 1);
        const real pszP = P.FA[2] + P.FB[2], pszC = C.FA[2] + C.FB[2];
        const real phzm = pszP + __shfl_down_sync(kFull, pszP, 1);
        const real phzp = pszC + __shfl_down_sync(kFull, pszC, 1);
        const real tR = __shfl_down_sync(kFull, P.tLo, 1);
        real so_sum = real(0), own = P.tLo;
        if constexpr (TT) {   // torso term, scattered with the domain flags
            const real qxm = (P.FAo[0] + C.FAo[0]) + (P.FBo[0] + C.FBo[0]);
            const real qxp = __shfl_down_sync(kFull, qxm, 1);
            const real qyA = P.FAo[1] + C.FAo[1], qyB = P.FBo[1] + C.FBo[1];
            const real qym = qyA + __shfl_down_sync(kFull, qyA, 1);
            const real qyp = qyB + __shfl_down_sync(kFull, qyB, 1);
            const real qzP = P.FAo[2] + P.FBo[2], qzC = C.FAo[2] + C.FBo[2];
            const real qzm = qzP + __shfl_down_sync(kFull, qzP, 1);
            const real qzp = qzC + __shfl_down_sync(kFull, qzC, 1);
            const real dR = __shfl_down_sync(kFull, P.dLo, 1);
            so_sum = P.dLoL * qxm - dR * qxp + P.dYm * qym - P.dHi * qyp + P.dzm * qzm - C.dLo * qzp;
            own = P.dLo;
        }
        bool mine = true;
        if constexpr (kGS<MODE>)   // this launch's colour only: (x & 1) + 2 (y & 1) + 4 (z & 1)
            mine = ((g.x & 1) | ((g.ylo & 1) << 1) | (((k - 1) & 1) << 2)) == o.colour;
        if (g.out_lane && own != real(0) && mine) {
            real s = P.tLoL * phxm - tR * phxp + P.tYm * phym - P.tHi * phyp + P.tzm * phzm - C.tLo * phzp;
            if constexpr (TT) s = P.tLo * s + so_sum;   // the tissue term acts on tissue voxels only
            const real Lu = o.C * s;
            const int q = g.qlo + (k - 1) * g.plane;
            if (MODE == M_APPLY || MODE == M_APPLY_BATH) {
                o.out[q] = Lu;
            } else if (MODE == M_RHS) {
                o.out[q] = -Lu;
            } else if (kJac<MODE>) {
                const real r = P.e0 - Lu;
                if (o.cform & kRestart) {   // correction form, first sweep of a cycle
                    if (o.cform & kFold) I.x0[q] += P.uLo;
                    I.b[q] = r;
                    o.out[q] = o.coef * P.e1 * r;
                } else {
                    const real basic = P.uLo + o.coef * P.e1 * r;
                    if (kCheb<MODE> && o.cheb) {   // x_{k+1} = w (basic - x_{k-1}) + x_{k-1}; x_{k-1} came through the ring
                        const real prev = (o.cform & kPrev0) ? real(0) : P.e2;
                        o.out[q] = o.cheb_w * (basic - prev) + prev;
                    } else {
                        o.out[q] = basic;
                    }
                }
                if (check) acc += (float)r * (float)r;
            } else if (MODE == M_IE) {   // r = f - (I + a L) x;  x+ = x + r / (1 + a D)  (Eq. iejac1)
                const real r = P.e0 - P.uLo - o.coef * Lu;
                o.out[q] = P.uLo + P.e1 * r;
                if (check) acc += (float)r * (float)r;
            } else if (MODE == M_IE_RHS) {
                o.out[q] = P.e0 - o.coef * Lu;   // f = v* - a L_i ve
                o.out2[q] = P.e0;                // first iterate: v*
                o.wout[q] = P.e1;
            } else {
                const real vnew = P.e0 - o.coef * Lu;
                o.out[q] = vnew;
                o.wout[q] = P.e1;
                const real vold = P.e2;
                if (vold < real(0.5) && vnew >= real(0.5)) {
                    const real t0 = o.tact[q];
                    if (t0 < real(0))
                        o.tact[q] = (real)(o.tn + o.dt_d * (0.5 - (double)vold) / ((double)vnew - (double)vold));
                }
                if (!isfinite((double)vnew)) atomicOr(&I.ctl->nonfinite, 1);
            }
        }
    }
}

template <typename real>
__device__ __forceinline__ void zero_state(St<real> &S)
{
    S.uLo = S.uHi = S.uLoL = S.uHiL = S.tLo = S.tHi = S.tLoL = S.tHiL = S.nT = real(0);
#pragma unroll
    for (int j = 0; j < 6; ++j) S.Y[j] = real(0);
    S.sx = S.cx = S.sy = S.cy = S.tYm = S.tzm = S.e0 = S.e1 = S.e2 = real(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) S.FB[j] = S.FA[j] = S.FBo[j] = S.FAo[j] = real(0);
    S.dLo = S.dHi = S.dLoL = S.dHiL = S.nB = S.sxd = S.cxd = S.syd = S.cyd = S.dYm = S.dzm = real(0);
}

// The Jacobi sweep and the monodomain step stage their loads through a
// per-thread ring in shared memory filled by cp.async D - 1 planes ahead:
// each thread reads back only what it copied itself, so the ring needs no
// barrier, and the prefetched planes hold no registers.  The other modes run
// once per step and prefetch one plane into registers.
// (The FP64 torso sweep prefetches into registers: its ring would not fit in
// 48 KB of static shared memory next to both terms' flux exchange.)
template <typename real, int MODE>
constexpr bool kRinged = (kJac<MODE> || MODE == M_IE || MODE == M_PAR_MONO) &&
                         !(kTwoTerm<MODE> && sizeof(real) == 8);

template <typename real, int MODE>
struct Ring {
    static constexpr int D = sizeof(real) == 4 ? 4 : 2;   // divides the unroll of 4; static smem < 48 KB
    static constexpr int NX = 2;   // b and x_{k-1} (Chebyshev) of row lo (Jacobi sweep), f and 1/(1+aD) of
                                   // row lo (implicit sweep), or w of rows lo, hi (monodomain step)
    float4 rec[D][2][kThreads];  // records of rows lo / hi
    real u[D][2][kThreads];
    real x[D][NX][kThreads];
};
struct NoRing {};

struct NoTorso {};

template <typename real, int MODE>
struct StencilSmem {
    real sF[2][3][kWarps][32];
    real sT[2][kWarps][32];
    double sred[kWarps];
    double cheb_w;   // Chebyshev weight of the sweep, formed by one thread (FP64 is slow here)
    int sflag;
    typename std::conditional<kRinged<real, MODE>, Ring<real, MODE>, NoRing>::type ring;
    typename std::conditional<kTwoTerm<MODE>, TorsoSmem<real>, NoTorso>::type tor;
};

// Bytes of shared memory of a stencil CTA (dynamic: with the ring and fp32 records the
// larger instances exceed the 48 KB of static shared memory; the host raises the limit).
template <typename real, int MODE>
constexpr size_t kSmemBytes = sizeof(StencilSmem<real, MODE>);

// The dynamic shared memory of the launch, as an object of type T.
template <typename T>
__device__ __forceinline__ T &dyn_smem()
{
    extern __shared__ __align__(16) unsigned char ep_dyn_smem[];
    return *reinterpret_cast<T *>(ep_dyn_smem);
}

template <int BYTES>
__device__ __forceinline__ void cp_async_n(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Stage plane k of this thread's two voxels into ring slot `slot`; off the
// grid the slot gets the values load_plane uses there.
template <typename real, int MODE>
__device__ __forceinline__ void ring_issue(const Op<real> &o, Ring<real, MODE> &R, int slot, int k, bool lo_in,
                                           bool hi_in, int qlo, int qhi, int plane)
{
    const int t = threadIdx.x;
    const bool kin = (unsigned)k < (unsigned)o.nz;
    if (kin && lo_in) {
        const int q = qlo + k * plane;
        cp_async_n<16>(&R.rec[slot][0][t], o.rec + q);
        cp_async_n<sizeof(real)>(&R.u[slot][0][t], o.src + q);
        cp_async_n<sizeof(real)>(&R.x[slot][0][t], (MODE == M_PAR_MONO ? o.w : o.b) + q);
        if (MODE == M_IE) cp_async_n<sizeof(real)>(&R.x[slot][1][t], o.inv + q);
        // x_{k-1} sits where this thread will write x_{k+1} of this voxel, one plane later
        if (kCheb<MODE> && o.cheb) cp_async_n<sizeof(real)>(&R.x[slot][1][t], o.out + q);
    } else {
        R.rec[slot][0][t] = make_float4(0.f, 0.f, 0.f, kNonTissueW);
        R.u[slot][0][t] = real(0);
        R.x[slot][0][t] = MODE == M_PAR_MONO ? real(1) : real(0);
        if (MODE == M_IE || kCheb<MODE>) R.x[slot][1][t] = real(0);
    }
    if (kin && hi_in) {
        const int q = qhi + k * plane;
        cp_async_n<16>(&R.rec[slot][1][t], o.rec + q);
        cp_async_n<sizeof(real)>(&R.u[slot][1][t], o.src + q);
        if (MODE == M_PAR_MONO) cp_async_n<sizeof(real)>(&R.x[slot][Ring<real, MODE>::NX - 1][t], o.w + q);
    } else {
        R.rec[slot][1][t] = make_float4(0.f, 0.f, 0.f, kNonTissueW);
        R.u[slot][1][t] = real(0);
        if (MODE == M_PAR_MONO) R.x[slot][Ring<real, MODE>::NX - 1][t] = real(1);
    }
}

template <typename real, int MODE>
__device__ __forceinline__ void ring_read(const Ring<real, MODE> &R, int slot, Ld<real, MODE> &L, bool o_cheb)
{
    const int t = threadIdx.x;
    L.rLo = R.rec[slot][0][t];
    L.rHi = R.rec[slot][1][t];
    L.uLo = R.u[slot][0][t];
    L.uHi = R.u[slot][1][t];
    if (kJac<MODE> || MODE == M_IE) {
        L.bLo = R.x[slot][0][t];
        L.iLo = (MODE == M_IE || (kCheb<MODE> && o_cheb)) ? R.x[slot][1][t] : real(0);
        L.wLo = L.wHi = real(1);
    } else {
        L.bLo = real(0);
        L.wLo = R.x[slot][0][t];
        L.wHi = R.x[slot][Ring<real, MODE>::NX - 1][t];
    }
    L.veLo = L.veHi = real(0);
}

// One plane: stage plane k + D - 1, wait for plane k (ring slot S % D), process it.
template <typename real, int MODE, int S>
__device__ __forceinline__ void ring_plane(const Inst<real> &I, const Op<real> &o, const Lane &g, int k, int kbeg,
                                           int kend, bool lo_in, bool hi_in, int qhi, Ring<real, MODE> &R,
                                           const St<real> &P, St<real> &Cn, Ld<real, MODE> &L,
                                           real (*sF)[3][kWarps][32], real (*sT)[kWarps][32], TorsoSmem<real> *ts,
                                           bool check, float &acc)
{
    constexpr int D = Ring<real, MODE>::D;
    constexpr int slot = S % D, next = (S + D - 1) % D;
    if (k + D - 1 <= kend) ring_issue<real, MODE>(o, R, next, k + D - 1, lo_in, hi_in, g.qlo, qhi, g.plane);
    cp_async_commit();
    cp_async_wait<D - 1>();
    ring_read<real, MODE>(R, slot, L, o.cheb != 0);
    plane_step<real, MODE>(I, o, g, k, k > kbeg, k > kbeg + 1, P, Cn, L, sF, sT, ts, check, acc);
}

// End of a sweep's work item: count its arrival; on a checking sweep the item
// that arrives last sums the FP64 partial norms in a fixed order and decides
// the stop (converged, diverged, non-finite) in the control block.
// (unit: the launch's index in the solve's launches, a sweep or, for the
// eight-colour sweep, a colour pass; parts: launches whose partial sums make up
// one sweep's residual, 1 or 8, and part this launch's place among them.)
template <typename real>
__device__ __forceinline__ void sweep_finish(const Inst<real> &I, int sweep, int unit, int part, int parts,
                                             int item, int nitems, bool check, bool eform, float acc, double *sred,
                                             int *sflag)
{
    Ctl *ctl = I.ctl;
    if (!check) {   // count the arrival; nobody waits on it within this launch
        if (threadIdx.x == 0) atomicAdd(&ctl->jarrive, 1ull);
        return;
    }
    // residual norm of this sweep's input: per-thread FP32 partial over its few voxels,
    // FP64 above; deterministic fixed-order reduction by the item that arrives last
    // (of the sweep's last launch)
    const double tot = block_sum<kThreads>((double)acc, sred);
    if (threadIdx.x == 0) {
        I.partials[part * nitems + item] = tot;
        __threadfence();
        const unsigned long long last = (unsigned long long)(unit + 1) * (unsigned long long)nitems - 1ull;
        *sflag = atomicAdd(&ctl->jarrive, 1ull) == last && part == parts - 1;
    }
    __syncthreads();
    if (*sflag) {
        __threadfence();
        double s = 0;
        for (int i = threadIdx.x; i < parts * nitems; i += kThreads) s += ((volatile double *)I.partials)[i];
        s = block_sum<kThreads>(s, sred);
        if (threadIdx.x == 0) {
            const int j = sweep + 1;
            ctl->sweep = j;
            ctl->rnorm2 = s;
            if (!(s == s) || isinf(s)) {
                ctl->nonfinite = 1; ctl->done = 1; ctl->iters = j;
            } else if (s <= ctl->thresh2) {
                ctl->converged = 1; ctl->done = 1; ctl->iters = j;
            } else if (s > I.div_factor * ctl->bnorm2) {
                ctl->diverged = 1; ctl->noconv = 1; ctl->done = 1; ctl->iters = j;
            } else if (eform) {   // correction form: sweep 0 starts the first cycle; a cycle that
                if (sweep == 0) {  // has cut ||r|| by 1e3 restarts at the next sweep
                    ctl->r0n2 = s;
                } else if (s <= kRestart2 * ctl->r0n2) {
                    ctl->cycle0 = j;
                    ctl->r0n2 = s;
                }
            }
            __threadfence();
        }
        __syncthreads();
    }
}

// One work item (segment) of one instance.  item / nitems: index of this item
// among the instance's items of the launch and their count (last-item logic).
// Returns false for a sweep of an instance whose solve is finished.
template <typename real, int MODE>
__device__ __forceinline__ void stencil_item(const Inst<real> &I, int seg_index, int item, int nitems,
                                             const ApplyIO<real> *io, StencilSmem<real, MODE> &sm)
{
    real(*sF)[3][kWarps][32] = reinterpret_cast<real(*)[3][kWarps][32]>(&sm.sF[0][0][0][0]);
    real(*sT)[kWarps][32] = reinterpret_cast<real(*)[kWarps][32]>(&sm.sT[0][0][0]);
    TorsoSmem<real> *ts = nullptr;
    if constexpr (kTwoTerm<MODE>) ts = &sm.tor;
    Ctl *ctl = I.ctl;

    Op<real> o;
    o.rec = I.rec;
    o.nz = I.nz;
    o.C = I.C;
    o.w = o.ve = o.b = o.inv = nullptr;
    o.out = o.wout = o.tact = o.out2 = nullptr;
    o.cheb = 0;
    o.cheb_w = real(1);
    o.cform = 0;
    o.colour = 0;
    o.so = I.sig_o;
    o.tn = 0.0;
    o.dt_d = I.dt_d;
    int sweep = 0, unit = 0;
    bool check = false;
    const long long step = (MODE == M_APPLY || MODE == M_APPLY_BATH) ? 0 : ctl->step;
    const int cur = (int)(step & 1);
    if (kSweep<MODE>) {
        unit = (int)(*(volatile unsigned long long *)&ctl->jarrive / (unsigned long long)nitems);
        sweep = unit;
        if (kGS<MODE>) {   // eight launches a sweep: colour pass unit & 7 of sweep unit >> 3
            sweep = unit >> 3;
            o.colour = unit & 7;
        }
        if (sweep >= I.max_iter) {   // sweep cap reached: the solve ends with the last iterate
            if (threadIdx.x == 0) {
                ctl->noconv = 1;
                ctl->iters = sweep;
                __threadfence();
                ctl->done = 1;
            }
            return;
        }
        if (kGS<MODE>) {   // in place: a colour's voxels are coupled to none of their own colour
            o.src = I.x0;
            o.out = I.x0;
            o.sT = I.sTie; o.dS = I.dSie; o.coef = I.coef_jac;
        } else if (kJac<MODE>) {
            o.src = (sweep & 1) ? I.x1 : I.x0;
            o.out = (sweep & 1) ? I.x0 : I.x1;
            o.sT = I.sTie; o.dS = I.dSie; o.coef = I.coef_jac;
            int kc = sweep;   // index of the sweep in its cycle (the semi-iteration's index)
            if (I.eform) {
                // correction form: the iterate is x0 + e; sweep 0 reads x0 itself (e_0 = 0 and
                // b - A x0 is the first cycle's right-hand side), later sweeps read e
                kc = sweep - *(volatile int *)&ctl->cycle0;
                if (sweep > 0) {
                    o.src = (sweep & 1) ? I.x1 : I.x2;
                    o.out = (sweep & 1) ? I.x2 : I.x1;
                }
                o.cform = (kc == 0 ? kRestart : 0) | (kc == 0 && sweep > 0 ? kFold : 0) | (kc == 1 ? kPrev0 : 0);
            }
            if (kCheb<MODE>) {   // the launch matches the descriptor's solver (host)
                o.coef = I.cheb_tau_c;
                if (kc > 0) {   // the first sweep of a cycle is the basic step itself
                    if (threadIdx.x == 0) sm.cheb_w = cheb_weight(kc, I.cheb_rho, I.cheb_theta);
                    __syncthreads();
                    o.cheb = 1;
                    o.cheb_w = (real)sm.cheb_w;
                }
            }
        } else {   // implicit sweep: iterates in the new v buffer and ie_x
            o.src = (sweep & 1) ? I.ie_x : I.v[cur ^ 1];
            o.out = (sweep & 1) ? I.v[cur ^ 1] : I.ie_x;
            o.inv = I.ie_inv;
            o.sT = I.sTi; o.dS = I.dSi; o.coef = I.alpha_ie;
        }
        o.b = I.b;
        check = (sweep % I.check_every) == 0;
    } else if (MODE == M_IE_RHS) {
        o.src = I.v[cur];
        o.w = I.w[cur];
        o.ve = I.x0;
        o.out = I.b;
        o.out2 = I.v[cur ^ 1];
        o.wout = I.w[cur ^ 1];
        o.sT = I.sTi; o.dS = I.dSi; o.coef = I.alpha_ie;
        o.tn = (double)step * I.dt_d;
    } else if (MODE == M_RHS) {
        o.src = I.v[cur ^ 1];        // v of step n + 1 (the step counter moves at the end of the step)
        o.out = I.b;
        o.sT = I.sTi; o.dS = I.dSi; o.coef = real(0);
    } else if (MODE == M_APPLY || MODE == M_APPLY_BATH) {
        o.src = io->u;
        o.out = io->out;
        o.sT = io->sT; o.dS = io->dS; o.coef = real(0);
    } else {
        o.src = I.v[cur];
        o.w = I.w[cur];
        o.ve = I.x0;
        o.out = I.v[cur ^ 1];
        o.wout = I.w[cur ^ 1];
        o.tact = I.tact;
        o.sT = I.sTi; o.dS = I.dSi; o.coef = I.coef_par;
        o.tn = (double)step * I.dt_d;
    }

    Lane g;
    g.lane = threadIdx.x & 31;
    g.wid = threadIdx.x >> 5;
    const Seg sg = I.segs[seg_index];
    g.x = sg.x0 - 1 + g.lane;
    g.ylo = sg.by * kTileY + g.wid - 1;
    const bool xin = g.x >= 0 && g.x < I.nx;
    const bool lo_in = xin && g.ylo >= 0 && g.ylo < I.ny;
    const bool hi_in = xin && g.ylo + 1 >= 0 && g.ylo + 1 < I.ny;
    g.plane = I.nx * I.ny;
    g.qlo = lo_in ? g.x + I.nx * g.ylo : 0;
    const int qhi = hi_in ? g.x + I.nx * (g.ylo + 1) : 0;
    g.out_lane = g.lane >= 1 && g.lane <= kTileX && g.wid >= 1 && lo_in;

    float acc = 0.f;
    St<real> S0, S1;
    zero_state(S0);
    zero_state(S1);
    Ld<real, MODE> L0, L1;
    const int kbeg = sg.k0 - 1, kend = sg.k1;
    if constexpr (kRinged<real, MODE>) {
        // planes staged D - 1 ahead through the shared-memory ring; the loop is
        // unrolled by 4 so that every ring slot is a compile-time constant
        constexpr int D = Ring<real, MODE>::D;
        Ring<real, MODE> &R = sm.ring;
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
            if (kbeg + j <= kend) ring_issue<real, MODE>(o, R, j, kbeg + j, lo_in, hi_in, g.qlo, qhi, g.plane);
            cp_async_commit();
        }
        for (int k = kbeg;;) {
            ring_plane<real, MODE, 0>(I, o, g, k, kbeg, kend, lo_in, hi_in, qhi, R, S1, S0, L0, sF, sT, ts, check, acc);
            if (++k > kend) break;
            ring_plane<real, MODE, 1>(I, o, g, k, kbeg, kend, lo_in, hi_in, qhi, R, S0, S1, L1, sF, sT, ts, check, acc);
            if (++k > kend) break;
            ring_plane<real, MODE, 2>(I, o, g, k, kbeg, kend, lo_in, hi_in, qhi, R, S1, S0, L0, sF, sT, ts, check, acc);
            if (++k > kend) break;
            ring_plane<real, MODE, 3>(I, o, g, k, kbeg, kend, lo_in, hi_in, qhi, R, S0, S1, L1, sF, sT, ts, check, acc);
            if (++k > kend) break;
        }
        cp_async_wait<0>();
    } else {
        load_plane<real, MODE>(o, kbeg, lo_in, hi_in, g.qlo, qhi, g.plane, L0);
        // two planes per iteration; the state records swap roles
        for (int k = kbeg;;) {
            if (k + 1 <= kend) load_plane<real, MODE>(o, k + 1, lo_in, hi_in, g.qlo, qhi, g.plane, L1);
            plane_step<real, MODE>(I, o, g, k, k > kbeg, k > kbeg + 1, S1, S0, L0, sF, sT, ts, check, acc);
            if (++k > kend) break;
            if (k + 1 <= kend) load_plane<real, MODE>(o, k + 1, lo_in, hi_in, g.qlo, qhi, g.plane, L0);
            plane_step<real, MODE>(I, o, g, k, k > kbeg, k > kbeg + 1, S0, S1, L1, sF, sT, ts, check, acc);
            if (++k > kend) break;
        }
    }

    if (kGS<MODE>)
        sweep_finish<real>(I, sweep, unit, o.colour, 8, item, nitems, check, false, acc, sm.sred, &sm.sflag);
    else if (kSweep<MODE>)
        sweep_finish<real>(I, sweep, sweep, 0, 1, item, nitems, check, kJac<MODE> && I.eform, acc, sm.sred,
                           &sm.sflag);
}

// Whether the solve of `ctl` is finished, read once for the whole CTA: a capped
// solve sets its flag while other CTAs of the same launch may be starting, and
// threads of one CTA that read it at different moments would part ways (in the
// batched kernels some of them would then miss their share of the descriptor
// copy).  Ends with a barrier.
__device__ __forceinline__ bool cta_done(const Ctl *ctl, int *sflag)
{
    if (threadIdx.x == 0) *sflag = *(const volatile int *)&ctl->done;
    __syncthreads();
    return *sflag != 0;
}

// Single instance: one CTA per segment.  The two-term modes keep both terms'
// vertex state and run two CTAs an SM.
template <typename real, int MODE>
__global__ void __launch_bounds__(kThreads, kTwoTerm<MODE> ? 2 : kMinBlocks) k_stencil(Inst<real> I, ApplyIO<real> io)
{
    StencilSmem<real, MODE> &sm = dyn_smem<StencilSmem<real, MODE>>();
    if (kSweep<MODE> && cta_done(I.ctl, &sm.sflag)) return;   // converged earlier: queued sweeps are no-ops
    const int nitems = I.nitems_all > 0 ? I.nitems_all : (int)gridDim.x;
    stencil_item<real, MODE>(I, blockIdx.x, I.item0 + (int)blockIdx.x, nitems, &io, sm);
}

// Copies a member's descriptor into shared memory (read there, like the
// by-value parameter of the single-instance kernel, instead of from global
// memory through a pointer the compiler must keep live).
template <typename real>
__device__ __forceinline__ const Inst<real> &stage_inst(const Inst<real> *src, Inst<real> &dst)
{
    static_assert(sizeof(Inst<real>) % 8 == 0, "descriptor copied in 8-byte words");
    const unsigned long long *a = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Inst<real>) / 8); i += blockDim.x) d[i] = a[i];
    __syncthreads();
    return dst;
}

// Batched: one CTA per entry of the packed (instance, item) list of all
// instances, so the hardware balances uneven items as in the single-instance
// launch; items of instances whose solve is finished return at once.
template <typename real, int MODE>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
k_stencil_batch(const Inst<real> *insts, const BItem *items)
{
    StencilSmem<real, MODE> &sm = dyn_smem<StencilSmem<real, MODE>>();
    __shared__ Inst<real> sI;
    const BItem it = items[blockIdx.x];
    if (kJac<MODE> && cta_done(insts[it.inst].ctl, &sm.sflag)) return;
    const Inst<real> &I = stage_inst(insts + it.inst, sI);
    stencil_item<real, MODE>(I, it.item, it.item, it.nitems, nullptr, sm);
}

// Batched sweeps over the unfinished members only (the list is rebuilt at
// every convergence check): CTA i takes item i - act[k].cum of member k,
// act[k].cum <= i < act[k + 1].cum, found by one parallel lookup over the
// entries of the group's n members (the list has n + 1 entries); a CTA that
// matches none (i past the total) returns.  The
// descriptor and the control block are then fetched together, so a CTA waits
// on three dependent loads before its data (the single-instance kernel, two).
template <typename real, int MODE>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
k_stencil_active(const Inst<real> *insts, const ActRec *act, int n)
{
    StencilSmem<real, MODE> &sm = dyn_smem<StencilSmem<real, MODE>>();
    __shared__ Inst<real> sI;
    __shared__ int sk;
    const int i = blockIdx.x;
    if (threadIdx.x == 0) sk = -1;
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const ActRec a = act[k];
        if (a.inst >= 0 && a.cum <= i && i < act[k + 1].cum) sk = k;   // at most one entry matches
    }
    __syncthreads();
    if (sk < 0) return;
    const ActRec r = act[sk];
    if (kJac<MODE> && cta_done(r.ctl, &sm.sflag)) return;   // converged at a check in this loop pass
    const Inst<real> &I = stage_inst(insts + r.inst, sI);
    const int item = i - r.cum;
    stencil_item<real, MODE>(I, item, item, I.nseg, nullptr, sm);
}

}  // namespace gbep
