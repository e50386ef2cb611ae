// Device code of the constant-coefficient modal stage shared by the
// per-problem kernels (gdg_const.cu) and the batched kernels (gdg_batch.cu).
#pragma once

#include "gdg_checks.cuh"
#include "gdg_internal.h"

namespace {



// trace buffer index: 2-D [e][face 0..3 = xm,xp,ym,yp][field 0 = v, 1 = n.grad u][N1]
// (signed: on a partitioned mesh the ghost row below the first row has e < 0)
template <int N1>
__device__ __forceinline__ long long tix2(int e, int face, int fld, int i) {
    return (((long long)e * 4 + face) * 2 + fld) * N1 + i;
}
// 1-D: [e][face 0..1][field]
__device__ __forceinline__ size_t tix1(int e, int face, int fld) {
    return ((size_t)e * 2 + face) * 2 + fld;
}

// Fluxes of Section 2.2.1 in normal form (alpha = 1/2):
//   v* = (vi + vo)/2 - beta (di + do),  q* = (di - do)/2 - tau (vi - vo)
// returns g = v* - vi and c2 * q*.  Alternating flux (alpha = 1, sides by a
// fixed orientation: side 1 = the left / lower element): on the element's
// minus face (side = 0, it is side 2) v* = vo, q* = di; on its plus face
// (side = 1) v* = vi, q* = -do; on a Dirichlet side (bnd: vo, do are the
// mirror state) v* = 0, q* = di, which is the alpha = 1/2 formula there.
__device__ __forceinline__ void flux(double vi, double di, double vo, double dO, double beta,
                                     double tau, double c2, int alt, int side, bool bnd, double &g, double &q) {
    if (alt && !bnd) {
        g = side == 0 ? vo - vi : 0.0;
        q = c2 * (side == 0 ? di : -dO);
        return;
    }
    g = 0.5 * (vo - vi) - beta * (di + dO);
    q = c2 * (0.5 * (di - dO) - tau * (vi - vo));
}

// The same fluxes doubled, without c^2 (g2 = 2 (v* - vi), q2 = 2 q*), as the
// parity stage bodies use them.
__device__ __forceinline__ void flux2(double vi, double di, double vo, double dO, double b2, double t2,
                                      int alt, int side, bool bnd, double &g2, double &q2) {
    const double d1 = vo - vi;
    if (alt && !bnd) {
        g2 = side == 0 ? 2.0 * d1 : 0.0;
        q2 = side == 0 ? 2.0 * di : -2.0 * dO;
        return;
    }
    g2 = fma(-b2, di + dO, d1);
    q2 = fma(t2, d1, di - dO);
}

// Body of the parity stage kernel for element tile `etile` (blockDim.x / N1
// elements per block).  Parity version of the generic stage: the GD element is symmetric under r -> 1-r,
// so every modified-basis vector is even or odd: Psi[N-i][k] = s_k Psi[i][k].
// With the NE = (N1+1)/2 even modes stored first, eR = s eL and gR = s gL:
// both face traces of a line come from one even/odd split dot, and each
// lift is one FMA per entry.  Fluxes carry a factor 2 (g2 = 2(v* - v_in),
// q2 = 2 q*) that is folded into the lift vectors hgL = gL/2, ceL = c^2 eL/2.
// ALT: the flux kind as a compile-time constant (1 alternating, 0 central or
// upwind; must equal mp.alt), so the per-face choice costs nothing.
// The u lifts enter only through k_u = V + Lambda^+ r_u, so they are folded
// with the diagonal solve: P1[l][k] = hgL_x[k] / lambda[l][k] and
// P2[l][k] = hgL_y[l] / lambda[l][k] (lam2 rows 2 and 3; 0 on the constant
// mode), two FMAs per entry.  RK4 accumulates k1 + 2 k2 + 2 k3 (stages 1-3
// ignore cA) and stage 4 forms y_n + cA (acc + k4) with cA = dt/6, the
// order of the classic formula y_n + dt/6 (k1 + 2 k2 + 2 k3 + k4).
template <int N1, int MODE, int ALT>
__device__ __forceinline__ void stage2p_body(const ModalParams &mp, const StageBufs &b, double cA, double cY,
                                             int etile, double *smem) {
    constexpr int NE = (N1 + 1) / 2;
    const int epb = blockDim.x / N1;
    const int t = threadIdx.x;
    const int le = t / N1, l = t - le * N1;
    const int e = etile * epb + le;
    const bool valid = le < epb && e < mp.ne;
    double *fy = smem + le * (4 * N1);   // per column: GA, GB, QA, QB of the y faces
    double *tile = smem + epb * 4 * N1 + le * (2 * N1 * (N1 + 1));
    const int nx = mp.nx, ny = mp.ny;
    const int ex = valid ? e % nx : 0, ey = valid ? e / nx : 0;
    const double b2 = mp.beta2, t2 = mp.tau2;
    const size_t row = ((size_t)(valid ? e : 0) * N1 + l) * N1;

    // issue every row load of this stage before the barrier so their latency
    // overlaps the flux work (a few warps per SM only at small element counts)
    double Ru[N1], Rv[N1], Nu[N1], Nv[N1], Au[N1], Av[N1];
    if (valid) {
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            Ru[k] = b.yU[row + k];
            Rv[k] = b.yV[row + k];
            if (MODE == M_S23 || MODE == M_S4) {
                Nu[k] = b.nU[row + k];
                Nv[k] = b.nV[row + k];
                Au[k] = b.aU[row + k];
                Av[k] = b.aV[row + k];
            }
        }
    }

    double GA = 0, GB = 0, QA = 0, QB = 0;
    if (valid) {
        const double *T = b.trin;
        double vi, di, vo, dO, g2m, q2m, g2p, q2p;
        int en, f;
        bool bnd;
        // x faces, transverse mode l
        vi = T[tix2<N1>(e, 0, 0, l)]; di = T[tix2<N1>(e, 0, 1, l)];
        en = ex - 1;
        if (en < 0 && mp.per_x) en += nx;
        bnd = en < 0;
        if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2P_NB + 0); vo = T[tix2<N1>(f, 1, 0, l)]; dO = T[tix2<N1>(f, 1, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 0, bnd, g2m, q2m);
        vi = T[tix2<N1>(e, 1, 0, l)]; di = T[tix2<N1>(e, 1, 1, l)];
        en = ex + 1;
        if (en >= nx && mp.per_x) en -= nx;
        bnd = en >= nx;
        if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2P_NB + 1); vo = T[tix2<N1>(f, 0, 0, l)]; dO = T[tix2<N1>(f, 0, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 1, bnd, g2p, q2p);
        GA = g2m + g2p; GB = g2m - g2p; QA = q2m + q2p; QB = q2m - q2p;
        // y faces, transverse mode k = l (on a halo side the neighbour row's
        // traces sit in the ghost row en = -1 or en = ny of the trace buffer)
        vi = T[tix2<N1>(e, 2, 0, l)]; di = T[tix2<N1>(e, 2, 1, l)];
        en = ey - 1;
        if (en < 0 && mp.per_y) en += ny;
        bnd = en < 0 && !mp.halo_lo;
        if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2P_NB + 2); vo = T[tix2<N1>(f, 3, 0, l)]; dO = T[tix2<N1>(f, 3, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 0, bnd, g2m, q2m);
        vi = T[tix2<N1>(e, 3, 0, l)]; di = T[tix2<N1>(e, 3, 1, l)];
        en = ey + 1;
        if (en >= ny && mp.per_y) en -= ny;
        bnd = en >= ny && !mp.halo_hi;
        if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2P_NB + 3); vo = T[tix2<N1>(f, 2, 0, l)]; dO = T[tix2<N1>(f, 2, 1, l)]; }
        else { vo = -vi; dO = -di; }
        flux2(vi, di, vo, dO, b2, t2, ALT, 1, bnd, g2p, q2p);
        fy[l] = g2m + g2p; fy[N1 + l] = g2m - g2p;
        fy[2 * N1 + l] = q2m + q2p; fy[3 * N1 + l] = q2m - q2p;
    }
    __syncthreads();

    if (valid) {
        const double *L0 = b.lam2 + l * N1;
        const double *P1 = b.lam2 + 2 * N1 * N1 + l * N1, *P2 = b.lam2 + 3 * N1 * N1 + l * N1;
        const double cey = mp.d[1].ceL[l];
        const double *FG = fy + (l < NE ? 0 : N1);
        const double *FQ = fy + (l < NE ? 2 * N1 : 3 * N1);
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const double Yu = Ru[k], Yv = Rv[k];
            const double xg = k < NE ? GA : GB, xq = k < NE ? QA : QB;
            // k_u = V + Lambda^+ r_u with the rank-one lifts folded into P1, P2
            const double ku = fma(P1[k], xg, fma(P2[k], FG[k], Yv));
            const double rv = fma(L0[k], Yu, fma(mp.d[0].ceL[k], xq, cey * FQ[k]));
            const double kv = rv;
            if (MODE == M_RHS) {
                b.oU[row + k] = ku;
                b.oV[row + k] = kv;
            } else if (MODE == M_S1) {   // accumulator k1 + 2 k2 + 2 k3, scaled by dt/6 at stage 4
                b.aU[row + k] = ku;
                b.aV[row + k] = kv;
                Ru[k] = fma(cY, ku, Yu);
                Rv[k] = fma(cY, kv, Yv);
            } else if (MODE == M_S23) {
                b.aU[row + k] = fma(2.0, ku, Au[k]);
                b.aV[row + k] = fma(2.0, kv, Av[k]);
                Ru[k] = fma(cY, ku, Nu[k]);
                Rv[k] = fma(cY, kv, Nv[k]);
            } else {
                Ru[k] = fma(cA, Au[k] + ku, Nu[k]);
                Rv[k] = fma(cA, Av[k] + kv, Nv[k]);
            }
        }
        if (MODE != M_RHS) {
            double *dU = (MODE == M_S4) ? b.nU : b.oU;
            double *dV = (MODE == M_S4) ? b.nV : b.oV;
#pragma unroll
            for (int k = 0; k < N1; ++k) { dU[row + k] = Ru[k]; dV[row + k] = Rv[k]; }
        }
    }
    if (MODE == M_RHS) return;

    if (valid) {
        double ve = 0, vo_ = 0, de = 0, do_ = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            if (k < NE) { ve = fma(mp.d[0].eL[k], Rv[k], ve); de = fma(mp.d[0].gL[k], Ru[k], de); }
            else { vo_ = fma(mp.d[0].eL[k], Rv[k], vo_); do_ = fma(mp.d[0].gL[k], Ru[k], do_); }
            tile[l * (N1 + 1) + k] = Ru[k];
            tile[N1 * (N1 + 1) + l * (N1 + 1) + k] = Rv[k];
        }
        b.trout[tix2<N1>(e, 0, 0, l)] = ve + vo_;
        b.trout[tix2<N1>(e, 0, 1, l)] = de + do_;
        b.trout[tix2<N1>(e, 1, 0, l)] = ve - vo_;
        b.trout[tix2<N1>(e, 1, 1, l)] = de - do_;
    }
    __syncthreads();
    if (valid) {
        const int k = l;
        double ve = 0, vo_ = 0, de = 0, do_ = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const double u = tile[j * (N1 + 1) + k], v = tile[N1 * (N1 + 1) + j * (N1 + 1) + k];
            if (j < NE) { ve = fma(mp.d[1].eL[j], v, ve); de = fma(mp.d[1].gL[j], u, de); }
            else { vo_ = fma(mp.d[1].eL[j], v, vo_); do_ = fma(mp.d[1].gL[j], u, do_); }
        }
        b.trout[tix2<N1>(e, 2, 0, k)] = ve + vo_;
        b.trout[tix2<N1>(e, 2, 1, k)] = de + do_;
        b.trout[tix2<N1>(e, 3, 0, k)] = ve - vo_;
        b.trout[tix2<N1>(e, 3, 1, k)] = de - do_;
    }
}

// Half-line variant of stage2p_body: two threads per transverse line, lane
// pair (2m, 2m+1), the even one (h = 0) owning the NE even modes k < NE and
// the odd one (h = 1) the odd modes k >= NE.  Every floating-point operation
// is the one stage2p_body performs, in the same order, so the two bodies give
// bit-identical results; a pair swaps face fluxes and trace partial sums by
// one shuffle.  Twice the threads and half the registers per element: more
// warps per SM to hide FP64 and shared-memory latency on small meshes.
// blockDim.x = epb * 2 * N1 (even, so a pair never straddles a warp).
__device__ __forceinline__ unsigned pair_mask() {
    const int lanes = min(32, (int)blockDim.x - (int)(threadIdx.x & ~31u));
    return lanes >= 32 ? 0xffffffffu : ((1u << lanes) - 1u);
}

// LEAN: y_n and the RK accumulator are read where the update uses them
// instead of with the stage input (same operations and results; 40 fewer
// live registers at S23 / S4, for kernels held to a low register count).
template <int N1, int MODE, bool LEAN = false>
__device__ __forceinline__ void stage2h_body(const ModalParams &mp, const StageBufs &b, double cA, double cY,
                                             int etile, double *smem) {
    constexpr int NE = (N1 + 1) / 2;   // even modes; the odd half has N1 - NE <= NE entries
    const int epb = blockDim.x / (2 * N1);
    const int t = threadIdx.x;
    const int le = t / (2 * N1), rr = t - le * (2 * N1);
    const int l = rr >> 1, h = rr & 1;
    const int k0 = h ? NE : 0, nk = h ? N1 - NE : NE;
    const int e = etile * epb + le;
    const bool valid = le < epb && e < mp.ne;
    const unsigned mask = pair_mask();
    double *fy = smem + (le < epb ? le : 0) * (4 * N1);
    double *tile = smem + epb * 4 * N1 + (le < epb ? le : 0) * (2 * N1 * (N1 + 1));
    const int nx = mp.nx, ny = mp.ny;
    const int ex = valid ? e % nx : 0, ey = valid ? e / nx : 0;
    const double b2 = mp.beta2, t2 = mp.tau2;
    const size_t row = ((size_t)(valid ? e : 0) * N1 + l) * N1 + k0;

    double Ru[NE], Rv[NE], Nu[NE], Nv[NE], Au[NE], Av[NE];
    if (valid) {
#pragma unroll
        for (int kk = 0; kk < NE; ++kk) {
            if (kk < nk) {
                Ru[kk] = b.yU[row + kk];
                Rv[kk] = b.yV[row + kk];
                if (!LEAN && (MODE == M_S23 || MODE == M_S4)) {
                    Nu[kk] = b.nU[row + kk];
                    Nv[kk] = b.nV[row + kk];
                    Au[kk] = b.aU[row + kk];
                    Av[kk] = b.aV[row + kk];
                }
            }
        }
    }

    // fluxes: h = 0 the minus face, h = 1 the plus face of each direction
    double gx = 0, qx = 0, gy = 0, qy = 0;
    if (valid) {
        const double *T = b.trin;
        double vi, di, vo, dO;
        int en, f;
        bool bnd;
        if (h == 0) {   // x-, transverse mode l
            vi = T[tix2<N1>(e, 0, 0, l)]; di = T[tix2<N1>(e, 0, 1, l)];
            en = ex - 1;
            if (en < 0 && mp.per_x) en += nx;
            bnd = en < 0;
            if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2H_NB + 0); vo = T[tix2<N1>(f, 1, 0, l)]; dO = T[tix2<N1>(f, 1, 1, l)]; }
            else { vo = -vi; dO = -di; }
        } else {        // x+
            vi = T[tix2<N1>(e, 1, 0, l)]; di = T[tix2<N1>(e, 1, 1, l)];
            en = ex + 1;
            if (en >= nx && mp.per_x) en -= nx;
            bnd = en >= nx;
            if (!bnd) { f = ey * nx + en; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2H_NB + 1); vo = T[tix2<N1>(f, 0, 0, l)]; dO = T[tix2<N1>(f, 0, 1, l)]; }
            else { vo = -vi; dO = -di; }
        }
        flux2(vi, di, vo, dO, b2, t2, mp.alt, h, bnd, gx, qx);
        if (h == 0) {   // y-, transverse mode l
            vi = T[tix2<N1>(e, 2, 0, l)]; di = T[tix2<N1>(e, 2, 1, l)];
            en = ey - 1;
            if (en < 0 && mp.per_y) en += ny;
            bnd = en < 0;
            if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2H_NB + 2); vo = T[tix2<N1>(f, 3, 0, l)]; dO = T[tix2<N1>(f, 3, 1, l)]; }
            else { vo = -vi; dO = -di; }
        } else {        // y+
            vi = T[tix2<N1>(e, 3, 0, l)]; di = T[tix2<N1>(e, 3, 1, l)];
            en = ey + 1;
            if (en >= ny && mp.per_y) en -= ny;
            bnd = en >= ny;
            if (!bnd) { f = en * nx + ex; GDG_CHECK_ELEM2(f, mp, GDG_SITE_STAGE2H_NB + 3); vo = T[tix2<N1>(f, 2, 0, l)]; dO = T[tix2<N1>(f, 2, 1, l)]; }
            else { vo = -vi; dO = -di; }
        }
        flux2(vi, di, vo, dO, b2, t2, mp.alt, h, bnd, gy, qy);
    }
    const double ogx = __shfl_xor_sync(mask, gx, 1), oqx = __shfl_xor_sync(mask, qx, 1);
    const double ogy = __shfl_xor_sync(mask, gy, 1), oqy = __shfl_xor_sync(mask, qy, 1);
    // g2m, g2p of each direction in the order of stage2p_body
    const double g2mx = h ? ogx : gx, g2px = h ? gx : ogx, q2mx = h ? oqx : qx, q2px = h ? qx : oqx;
    const double g2my = h ? ogy : gy, g2py = h ? gy : ogy, q2my = h ? oqy : qy, q2py = h ? qy : oqy;
    // x fluxes of this half's parity (GA, QA even; GB, QB odd)
    const double xg = h ? g2mx - g2px : g2mx + g2px;
    const double xq = h ? q2mx - q2px : q2mx + q2px;
    if (valid) {
        if (h == 0) { fy[l] = g2my + g2py; fy[2 * N1 + l] = q2my + q2py; }
        else { fy[N1 + l] = g2my - g2py; fy[3 * N1 + l] = q2my - q2py; }
    }
    __syncthreads();

    if (valid) {
        const double *L0 = b.lam2 + l * N1 + k0;
        const double *P1 = b.lam2 + 2 * N1 * N1 + l * N1 + k0, *P2 = b.lam2 + 3 * N1 * N1 + l * N1 + k0;
        const double cey = mp.d[1].ceL[l];
        const double *FG = fy + (l < NE ? 0 : N1) + k0;
        const double *FQ = fy + (l < NE ? 2 * N1 : 3 * N1) + k0;
        const double *cex = mp.d[0].ceL + k0;
#pragma unroll
        for (int kk = 0; kk < NE; ++kk) {
            if (kk < nk) {
                const double Yu = Ru[kk], Yv = Rv[kk];
                const double ku = fma(P1[kk], xg, fma(P2[kk], FG[kk], Yv));
                const double rv = fma(L0[kk], Yu, fma(cex[kk], xq, cey * FQ[kk]));
                const double kv = rv;
                const size_t o = row + kk;
                if (LEAN && (MODE == M_S23 || MODE == M_S4)) {
                    Nu[kk] = b.nU[o];
                    Nv[kk] = b.nV[o];
                    Au[kk] = b.aU[o];
                    Av[kk] = b.aV[o];
                }
                if (MODE == M_RHS) {
                    b.oU[o] = ku;
                    b.oV[o] = kv;
                } else if (MODE == M_S1) {
                    b.aU[o] = ku;
                    b.aV[o] = kv;
                    Ru[kk] = fma(cY, ku, Yu);
                    Rv[kk] = fma(cY, kv, Yv);
                } else if (MODE == M_S23) {
                    b.aU[o] = fma(2.0, ku, Au[kk]);
                    b.aV[o] = fma(2.0, kv, Av[kk]);
                    Ru[kk] = fma(cY, ku, Nu[kk]);
                    Rv[kk] = fma(cY, kv, Nv[kk]);
                } else {
                    Ru[kk] = fma(cA, Au[kk] + ku, Nu[kk]);
                    Rv[kk] = fma(cA, Av[kk] + kv, Nv[kk]);
                }
            }
        }
        if (MODE != M_RHS) {
            double *dU = (MODE == M_S4) ? b.nU : b.oU;
            double *dV = (MODE == M_S4) ? b.nV : b.oV;
#pragma unroll
            for (int kk = 0; kk < NE; ++kk)
                if (kk < nk) { dU[row + kk] = Ru[kk]; dV[row + kk] = Rv[kk]; }
        }
    }
    if (MODE == M_RHS) return;

    // x-face traces: this half's partial dots (even: ve, de; odd: vo, do)
    double pv = 0, pd = 0;
    if (valid) {
        const double *eLx = mp.d[0].eL + k0, *gLx = mp.d[0].gL + k0;
#pragma unroll
        for (int kk = 0; kk < NE; ++kk) {
            if (kk < nk) {
                pv = fma(eLx[kk], Rv[kk], pv);
                pd = fma(gLx[kk], Ru[kk], pd);
                tile[l * (N1 + 1) + k0 + kk] = Ru[kk];
                tile[N1 * (N1 + 1) + l * (N1 + 1) + k0 + kk] = Rv[kk];
            }
        }
    }
    {
        const double opv = __shfl_xor_sync(mask, pv, 1), opd = __shfl_xor_sync(mask, pd, 1);
        const double ve = h ? opv : pv, de = h ? opd : pd, vo_ = h ? pv : opv, do_ = h ? pd : opd;
        if (valid) {
            if (h == 0) {
                b.trout[tix2<N1>(e, 0, 0, l)] = ve + vo_;
                b.trout[tix2<N1>(e, 0, 1, l)] = de + do_;
            } else {
                b.trout[tix2<N1>(e, 1, 0, l)] = ve - vo_;
                b.trout[tix2<N1>(e, 1, 1, l)] = de - do_;
            }
        }
    }
    __syncthreads();
    // y-face traces of column k = l: this half's rows j (even j < NE, odd j >= NE)
    pv = 0;
    pd = 0;
    if (valid) {
        const int k = l;
        const double *eLy = mp.d[1].eL + k0, *gLy = mp.d[1].gL + k0;
#pragma unroll
        for (int jj = 0; jj < NE; ++jj) {
            if (jj < nk) {
                const int j = k0 + jj;
                const double u = tile[j * (N1 + 1) + k], v = tile[N1 * (N1 + 1) + j * (N1 + 1) + k];
                pv = fma(eLy[jj], v, pv);
                pd = fma(gLy[jj], u, pd);
            }
        }
    }
    {
        const double opv = __shfl_xor_sync(mask, pv, 1), opd = __shfl_xor_sync(mask, pd, 1);
        const double ve = h ? opv : pv, de = h ? opd : pd, vo_ = h ? pv : opv, do_ = h ? pd : opd;
        if (valid) {
            const int k = l;
            if (h == 0) {
                b.trout[tix2<N1>(e, 2, 0, k)] = ve + vo_;
                b.trout[tix2<N1>(e, 2, 1, k)] = de + do_;
            } else {
                b.trout[tix2<N1>(e, 3, 0, k)] = ve - vo_;
                b.trout[tix2<N1>(e, 3, 1, k)] = de - do_;
            }
        }
    }
}

}  // namespace
