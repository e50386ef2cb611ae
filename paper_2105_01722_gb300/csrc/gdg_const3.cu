// 3-D elements on the modal route (the tensor-product construction of
// Sections 2.1.2 and 3 for d = 3; the paper states it and tests d <= 2):
// fused RK stage, traces, separable transforms and the energy partials of
// gdg_step / gdg_rhs / gdg_mass_solve / gdg_energy for dim = 3 contexts.
// Modal layout [e][m3][m2][m1] (m1 along x); one thread per x line (m3, m2)
// of an element, blockDim.x = epb * N1 * N1.
#include <algorithm>

#include "gdg_checks.cuh"
#include "gdg_internal.h"
#include "gdg_stage_const.cuh"

namespace {

constexpr int MAXB3 = 256;   // threads per block (epb elements x N1^2 lines)

// trace buffer index: [e][face 0..5 = xm,xp,ym,yp,zm,zp][field][N1*N1];
// transverse index: x faces m3*N1+m2, y faces m3*N1+m1, z faces m2*N1+m1
template <int N1>
__device__ __forceinline__ size_t tix3(int e, int face, int fld, int t) {
    return (((size_t)e * 6 + face) * 2 + fld) * (N1 * N1) + t;
}

// neighbour across face f of element (ex, ey, ez); -1 on a Dirichlet side
__device__ __forceinline__ int nbr3(const ModalParams &mp, int ex, int ey, int ez, int f) {
    int x = ex, y = ey, z = ez;
    switch (f) {
    case 0: x -= 1; if (x < 0) { if (!mp.per_x) return -1; x += mp.nx; } break;
    case 1: x += 1; if (x >= mp.nx) { if (!mp.per_x) return -1; x -= mp.nx; } break;
    case 2: y -= 1; if (y < 0) { if (!mp.per_y) return -1; y += mp.ny; } break;
    case 3: y += 1; if (y >= mp.ny) { if (!mp.per_y) return -1; y -= mp.ny; } break;
    case 4: z -= 1; if (z < 0) { if (!mp.per_z) return -1; z += mp.nz; } break;
    default: z += 1; if (z >= mp.nz) { if (!mp.per_z) return -1; z -= mp.nz; } break;
    }
    return (z * mp.ny + y) * mp.nx + x;
}

// traces on the y and z faces from the element tile (tU, tV in shared
// memory, [m3][m2][m1]); thread (a, c): y faces at (m3 = a, m1 = c), z faces
// at (m2 = a, m1 = c)
template <int N1>
__device__ __forceinline__ void traces3_yz(const ModalParams &mp, const double *tU, const double *tV, int e,
                                           int a, int c, double *trout) {
    double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
    for (int m2 = 0; m2 < N1; ++m2) {
        const double u = tU[(a * N1 + m2) * N1 + c], v = tV[(a * N1 + m2) * N1 + c];
        vL += mp.d[1].eL[m2] * v;
        vR += mp.d[1].eR[m2] * v;
        dL += mp.d[1].gL[m2] * u;
        dR += mp.d[1].gR[m2] * u;
    }
    const int ty = a * N1 + c;
    trout[tix3<N1>(e, 2, 0, ty)] = vL;
    trout[tix3<N1>(e, 2, 1, ty)] = dL;
    trout[tix3<N1>(e, 3, 0, ty)] = vR;
    trout[tix3<N1>(e, 3, 1, ty)] = dR;
    vL = vR = dL = dR = 0;
#pragma unroll
    for (int m3 = 0; m3 < N1; ++m3) {
        const double u = tU[(m3 * N1 + a) * N1 + c], v = tV[(m3 * N1 + a) * N1 + c];
        vL += mp.d[2].eL[m3] * v;
        vR += mp.d[2].eR[m3] * v;
        dL += mp.d[2].gL[m3] * u;
        dR += mp.d[2].gR[m3] * u;
    }
    trout[tix3<N1>(e, 4, 0, ty)] = vL;
    trout[tix3<N1>(e, 4, 1, ty)] = dL;
    trout[tix3<N1>(e, 5, 0, ty)] = vR;
    trout[tix3<N1>(e, 5, 1, ty)] = dR;
}

template <int N1>
__host__ __device__ constexpr int smem3_doubles() { return 12 * N1 * N1 + 2 * N1 * N1 * N1; }

// elements per block of the 3-D kernels (epb3 on the host)
template <int N1>
__host__ __device__ constexpr int epb3c() { return MAXB3 / (N1 * N1) > 1 ? MAXB3 / (N1 * N1) : 1; }

template <int N1, int MODE>
__global__ void __launch_bounds__(MAXB3)
k_stage3(const __grid_constant__ ModalParams mp, const StageBufs b, double cA, double cY) {
    constexpr int NT = N1 * N1, NA = N1 * N1 * N1;
    extern __shared__ double smem[];
    const int epb = blockDim.x / NT;
    const int t = threadIdx.x;
    const int le = t / NT, r = t - le * NT;
    const int a = r / N1, c = r - (r / N1) * N1;
    const int e = blockIdx.x * epb + le;
    const bool valid = e < mp.ne;
    double *F = smem + le * smem3_doubles<N1>();      // [12][NT]: g, q of faces 0..5
    double *tU = F + 12 * NT, *tV = tU + NA;
    const int ex = valid ? e % mp.nx : 0, ey = valid ? (e / mp.nx) % mp.ny : 0, ez = valid ? e / (mp.nx * mp.ny) : 0;

    if (valid) {   // fluxes of the six faces at this thread's transverse mode pair
        const double *T = b.trin;
        const int tt = a * N1 + c;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const double vi = T[tix3<N1>(e, f, 0, tt)], di = T[tix3<N1>(e, f, 1, tt)];
            int nb = nbr3(mp, ex, ey, ez, f);
            double vo, dO;
            if (nb >= 0) {
                GDG_CHECK_INDEX(nb, 0, mp.ne, GDG_SITE_STAGE3_NB + f, 0);
                vo = T[tix3<N1>(nb, f ^ 1, 0, tt)]; dO = T[tix3<N1>(nb, f ^ 1, 1, tt)];
            }
            else { vo = -vi; dO = -di; }
            double g, q;
            flux(vi, di, vo, dO, mp.beta, mp.tau, mp.c2, mp.alt, f & 1, nb < 0, g, q);
            F[(2 * f) * NT + tt] = g;
            F[(2 * f + 1) * NT + tt] = q;
        }
    }
    __syncthreads();

    double Ru[N1], Rv[N1];   // next stage input (or k) on line (m3 = a, m2 = c)
    if (valid) {
        const int line = a * N1 + c;
        const size_t row = ((size_t)e * NT + line) * N1;
        const double *L0 = b.lam2 + line * N1;
        const double *L1 = b.lam2 + NA + line * N1;
        const double Gxm = F[0 * NT + line], Qxm = F[1 * NT + line];
        const double Gxp = F[2 * NT + line], Qxp = F[3 * NT + line];
        const double gLy = mp.d[1].gL[c], gRy = mp.d[1].gR[c], eLy = mp.d[1].eL[c], eRy = mp.d[1].eR[c];
        const double gLz = mp.d[2].gL[a], gRz = mp.d[2].gR[a], eLz = mp.d[2].eL[a], eRz = mp.d[2].eR[a];
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const int ty = a * N1 + k, tz = c * N1 + k;
            const double Yu = b.yU[row + k], Yv = b.yV[row + k];
            const double ru = mp.d[0].gL[k] * Gxm + mp.d[0].gR[k] * Gxp + gLy * F[4 * NT + ty] +
                              gRy * F[6 * NT + ty] + gLz * F[8 * NT + tz] + gRz * F[10 * NT + tz];
            const double rv = L0[k] * Yu + mp.d[0].eL[k] * Qxm + mp.d[0].eR[k] * Qxp + eLy * F[5 * NT + ty] +
                              eRy * F[7 * NT + ty] + eLz * F[9 * NT + tz] + eRz * F[11 * NT + tz];
            const double ku = Yv + L1[k] * ru;
            const double kv = rv;
            if (MODE == M_RHS) {
                b.oU[row + k] = ku;
                b.oV[row + k] = kv;
            } else if (MODE == M_S1) {
                b.aU[row + k] = cA * ku;
                b.aV[row + k] = cA * kv;
                Ru[k] = Yu + cY * ku;
                Rv[k] = Yv + cY * kv;
            } else if (MODE == M_S23) {
                b.aU[row + k] += cA * ku;
                b.aV[row + k] += cA * kv;
                Ru[k] = b.nU[row + k] + cY * ku;
                Rv[k] = b.nV[row + k] + cY * kv;
            } else {
                Ru[k] = b.nU[row + k] + b.aU[row + k] + cA * ku;
                Rv[k] = b.nV[row + k] + b.aV[row + k] + cA * kv;
            }
        }
        if (MODE != M_RHS) {
            double *dU = (MODE == M_S4) ? b.nU : b.oU;
            double *dV = (MODE == M_S4) ? b.nV : b.oV;
#pragma unroll
            for (int k = 0; k < N1; ++k) { dU[row + k] = Ru[k]; dV[row + k] = Rv[k]; }
        }
    }
    if (MODE == M_RHS) return;   // uniform across the block

    if (valid) {   // x faces from the line; the tile for the y and z faces
        const int line = a * N1 + c;
        double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            vL += mp.d[0].eL[k] * Rv[k];
            vR += mp.d[0].eR[k] * Rv[k];
            dL += mp.d[0].gL[k] * Ru[k];
            dR += mp.d[0].gR[k] * Ru[k];
            tU[line * N1 + k] = Ru[k];
            tV[line * N1 + k] = Rv[k];
        }
        b.trout[tix3<N1>(e, 0, 0, line)] = vL;
        b.trout[tix3<N1>(e, 0, 1, line)] = dL;
        b.trout[tix3<N1>(e, 1, 0, line)] = vR;
        b.trout[tix3<N1>(e, 1, 1, line)] = dR;
    }
    __syncthreads();
    if (valid) traces3_yz<N1>(mp, tU, tV, e, a, c, b.trout);
}

// The u lifts are folded with the diagonal solve (rows 2-4 of lam2: hgL of
// each direction over lambda) and RK4 accumulates k1 + 2 k2 + 2 k3 (stages
// 1-3 ignore cA; stage 4 forms y_n + cA (acc + k4), cA = dt/6), as the 2-D
// parity kernels do.
// Parity version of k_stage3 (modes ordered even first in every direction:
// eR = s eL and gR = s gL, s = +1 for the NE = (N1+1)/2 even modes, -1 for
// the odd ones).  Phase 1 keeps, per direction and transverse mode pair, the
// sum and the difference of the doubled minus- and plus-face fluxes
// (flux2), so that each face pair lifts onto an entry with one product
// (hgL = gL/2, ceL = c^2 eL/2 carry the factors): 3 terms for r_u and 4 for
// r_v instead of 6 and 7.  Each trace pair comes from one dot split into its
// even and odd parts (left = even + odd, right = even - odd).
template <int N1>
__device__ __forceinline__ void traces3_yz_p(const ModalParams &mp, const double *tU, const double *tV, int e,
                                             int a, int c, double *trout) {
    constexpr int NE = (N1 + 1) / 2;
    double ve = 0, vo = 0, de = 0, dd = 0;
#pragma unroll
    for (int m2 = 0; m2 < N1; ++m2) {
        const double u = tU[(a * N1 + m2) * N1 + c], v = tV[(a * N1 + m2) * N1 + c];
        if (m2 < NE) { ve = fma(mp.d[1].eL[m2], v, ve); de = fma(mp.d[1].gL[m2], u, de); }
        else { vo = fma(mp.d[1].eL[m2], v, vo); dd = fma(mp.d[1].gL[m2], u, dd); }
    }
    const int ty = a * N1 + c;
    trout[tix3<N1>(e, 2, 0, ty)] = ve + vo;
    trout[tix3<N1>(e, 2, 1, ty)] = de + dd;
    trout[tix3<N1>(e, 3, 0, ty)] = ve - vo;
    trout[tix3<N1>(e, 3, 1, ty)] = de - dd;
    ve = vo = de = dd = 0;
#pragma unroll
    for (int m3 = 0; m3 < N1; ++m3) {
        const double u = tU[(m3 * N1 + a) * N1 + c], v = tV[(m3 * N1 + a) * N1 + c];
        if (m3 < NE) { ve = fma(mp.d[2].eL[m3], v, ve); de = fma(mp.d[2].gL[m3], u, de); }
        else { vo = fma(mp.d[2].eL[m3], v, vo); dd = fma(mp.d[2].gL[m3], u, dd); }
    }
    trout[tix3<N1>(e, 4, 0, ty)] = ve + vo;
    trout[tix3<N1>(e, 4, 1, ty)] = de + dd;
    trout[tix3<N1>(e, 5, 0, ty)] = ve - vo;
    trout[tix3<N1>(e, 5, 1, ty)] = de - dd;
}

template <int N1, int MODE, int ALT>
__global__ void __launch_bounds__(MAXB3, 3)
k_stage3p(const __grid_constant__ ModalParams mp, const StageBufs b, double cA, double cY) {
    constexpr int NT = N1 * N1, NA = N1 * N1 * N1, NE = (N1 + 1) / 2;
    constexpr int EPB = epb3c<N1>(), BD = EPB * NT;   // blockDim.x == BD (launch_stage3)
    extern __shared__ double smem[];
    const int t = threadIdx.x;
    const int le = t / NT, r = t - le * NT;
    const int a = r / N1, c = r - (r / N1) * N1;
    const int e = blockIdx.x * EPB + le;
    const bool valid = e < mp.ne;
    // per element [12][NT]: per direction d, at 4d: g-sum, g-difference,
    // q-sum, q-difference; then the tile tU, tV
    double *F = smem + le * smem3_doubles<N1>();
    double *tU = F + 12 * NT, *tV = tU + NA;
    double *ce = smem + EPB * smem3_doubles<N1>();   // [3][N1]: c^2 eL / 2 of x, y, z
    if (t < N1) { ce[t] = mp.d[0].ceL[t]; ce[N1 + t] = mp.d[1].ceL[t]; ce[2 * N1 + t] = mp.d[2].ceL[t]; }
    const int ex = valid ? e % mp.nx : 0, ey = valid ? (e / mp.nx) % mp.ny : 0, ez = valid ? e / (mp.nx * mp.ny) : 0;

    if (valid) {   // fluxes of the three face pairs at this thread's transverse mode pair
        const double *T = b.trin;
        const int tt = a * N1 + c;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double g2[2], q2[2];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int f = 2 * d + side;
                const double vi = T[tix3<N1>(e, f, 0, tt)], di = T[tix3<N1>(e, f, 1, tt)];
                int nb = nbr3(mp, ex, ey, ez, f);
                double vo, dO;
                if (nb >= 0) {
                    GDG_CHECK_INDEX(nb, 0, mp.ne, GDG_SITE_STAGE3_NB + f, 0);
                    vo = T[tix3<N1>(nb, f ^ 1, 0, tt)]; dO = T[tix3<N1>(nb, f ^ 1, 1, tt)];
                }
                else { vo = -vi; dO = -di; }
                flux2(vi, di, vo, dO, mp.beta2, mp.tau2, ALT, side, nb < 0, g2[side], q2[side]);
            }
            F[(4 * d + 0) * NT + tt] = g2[0] + g2[1];
            F[(4 * d + 1) * NT + tt] = g2[0] - g2[1];
            F[(4 * d + 2) * NT + tt] = q2[0] + q2[1];
            F[(4 * d + 3) * NT + tt] = q2[0] - q2[1];
        }
    }
    __syncthreads();

    // The update runs over the block's EPB N1^3 consecutive entries in a
    // coalesced order: thread t takes entries t + s BD (s < N1), so every
    // warp load and store of the state covers 32 consecutive doubles (one x
    // line per thread would stride them by N1).  Entry q = (m3 N1 + m2) N1 +
    // m1 of element le2 finds its line's fluxes in that element's F; each
    // entry's arithmetic is the same sequence of operations in either order.
    // The stage's arrays do not overlap: with restrict the next entry's loads
    // may be issued before this entry's stores.
    const double *__restrict__ pyU = b.yU, *__restrict__ pyV = b.yV;
    double *__restrict__ paU = b.aU, *__restrict__ paV = b.aV, *__restrict__ pnU = b.nU, *__restrict__ pnV = b.nV;
    double *__restrict__ poU = b.oU, *__restrict__ poV = b.oV;
    const double *__restrict__ lam = b.lam2;
    const size_t base = (size_t)blockIdx.x * EPB * NA;
#pragma unroll
    for (int s = 0; s < N1; ++s) {
        const int idx = t + s * BD;
        const int le2 = idx / NA, q = idx - le2 * NA;
        if (blockIdx.x * EPB + le2 >= mp.ne) continue;
        const int line = q / N1, k = q - line * N1;
        const int m3 = line / N1, m2 = line - m3 * N1;
        double *F2 = smem + le2 * smem3_doubles<N1>();
        const size_t g = base + idx;
        const double Yu = pyU[g], Yv = pyV[g];
        const double xg = F2[(k < NE ? 0 : 1) * NT + line], xq = F2[(k < NE ? 2 : 3) * NT + line];
        const double FGy = F2[(4 + (m2 < NE ? 0 : 1)) * NT + m3 * N1 + k];   // at ty = m3 N1 + m1
        const double FQy = F2[(6 + (m2 < NE ? 0 : 1)) * NT + m3 * N1 + k];
        const double FGz = F2[(8 + (m3 < NE ? 0 : 1)) * NT + m2 * N1 + k];   // at tz = m2 N1 + m1
        const double FQz = F2[(10 + (m3 < NE ? 0 : 1)) * NT + m2 * N1 + k];
        // k_u = V + Lambda^+ r_u with the three rank-one lifts folded into
        // rows 2-4 of lam2 (hgL / lambda per direction): three FMAs
        const double ku = fma(lam[2 * NA + q], xg, fma(lam[3 * NA + q], FGy, fma(lam[4 * NA + q], FGz, Yv)));
        const double rv = fma(lam[q], Yu, fma(ce[k], xq, fma(ce[N1 + m2], FQy, ce[2 * N1 + m3] * FQz)));
        const double kv = rv;
        double Ru, Rv;
        if (MODE == M_RHS) {
            poU[g] = ku;
            poV[g] = kv;
            continue;
        } else if (MODE == M_S1) {   // accumulator k1 + 2 k2 + 2 k3, scaled by dt/6 at stage 4
            paU[g] = ku;
            paV[g] = kv;
            Ru = fma(cY, ku, Yu);
            Rv = fma(cY, kv, Yv);
        } else if (MODE == M_S23) {
            paU[g] = fma(2.0, ku, paU[g]);
            paV[g] = fma(2.0, kv, paV[g]);
            Ru = fma(cY, ku, pnU[g]);
            Rv = fma(cY, kv, pnV[g]);
        } else {
            Ru = fma(cA, paU[g] + ku, pnU[g]);
            Rv = fma(cA, paV[g] + kv, pnV[g]);
        }
        if (MODE == M_S4) { pnU[g] = Ru; pnV[g] = Rv; }
        else { poU[g] = Ru; poV[g] = Rv; }
        double *tU2 = F2 + 12 * NT;
        tU2[q] = Ru;
        tU2[NA + q] = Rv;
    }
    if (MODE == M_RHS) return;   // uniform across the block
    __syncthreads();

    if (valid) {   // x faces from this thread's line; the tile for the y and z faces
        const int line = a * N1 + c;
        double ve = 0, vo = 0, de = 0, dd = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const double u = tU[line * N1 + k], v = tV[line * N1 + k];
            if (k < NE) { ve = fma(mp.d[0].eL[k], v, ve); de = fma(mp.d[0].gL[k], u, de); }
            else { vo = fma(mp.d[0].eL[k], v, vo); dd = fma(mp.d[0].gL[k], u, dd); }
        }
        b.trout[tix3<N1>(e, 0, 0, line)] = ve + vo;
        b.trout[tix3<N1>(e, 0, 1, line)] = de + dd;
        b.trout[tix3<N1>(e, 1, 0, line)] = ve - vo;
        b.trout[tix3<N1>(e, 1, 1, line)] = de - dd;
        traces3_yz_p<N1>(mp, tU, tV, e, a, c, b.trout);
    }
}

// traces of a modal state (start of gdg_step and gdg_rhs)
template <int N1>
__global__ void __launch_bounds__(MAXB3)
k_traces3(const __grid_constant__ ModalParams mp, const double *yU, const double *yV, double *trout) {
    constexpr int NT = N1 * N1, NA = N1 * N1 * N1;
    extern __shared__ double smem[];
    const int epb = blockDim.x / NT;
    const int t = threadIdx.x;
    const int le = t / NT, r = t - le * NT;
    const int a = r / N1, c = r - (r / N1) * N1;
    const int e = blockIdx.x * epb + le;
    const bool valid = e < mp.ne;
    double *tU = smem + le * 2 * NA, *tV = tU + NA;
    if (valid) {
        const int line = a * N1 + c;
        const size_t row = ((size_t)e * NT + line) * N1;
        double vL = 0, vR = 0, dL = 0, dR = 0;
#pragma unroll
        for (int k = 0; k < N1; ++k) {
            const double u = yU[row + k], v = yV[row + k];
            vL += mp.d[0].eL[k] * v;
            vR += mp.d[0].eR[k] * v;
            dL += mp.d[0].gL[k] * u;
            dR += mp.d[0].gR[k] * u;
            tU[line * N1 + k] = u;
            tV[line * N1 + k] = v;
        }
        trout[tix3<N1>(e, 0, 0, line)] = vL;
        trout[tix3<N1>(e, 0, 1, line)] = dL;
        trout[tix3<N1>(e, 1, 0, line)] = vR;
        trout[tix3<N1>(e, 1, 1, line)] = dR;
    }
    __syncthreads();
    if (valid) traces3_yz<N1>(mp, tU, tV, e, a, c, trout);
}

// Separable element transform out = (Cz (x) Cy (x) Cx) diag(D) (Bz (x) By (x) Bx) in
// (C, D optional); per field, passes along x, y, z through an element tile.
template <int N1>
__global__ void __launch_bounds__(MAXB3)
k_sep3(int ne, const double *in0, const double *in1, double *out0, double *out1, const double *Bx,
       const double *By, const double *Bz, const double *D, const double *Cx, const double *Cy, const double *Cz) {
    constexpr int NT = N1 * N1, NA = N1 * N1 * N1;
    extern __shared__ double smem[];
    double *sM = smem;            // Bx, By, Bz, Cx, Cy, Cz
    const int t = threadIdx.x;
    for (int i = t; i < NT; i += blockDim.x) {
        sM[i] = Bx[i];
        sM[NT + i] = By[i];
        sM[2 * NT + i] = Bz[i];
        if (Cx) { sM[3 * NT + i] = Cx[i]; sM[4 * NT + i] = Cy[i]; sM[5 * NT + i] = Cz[i]; }
    }
    const int epb = blockDim.x / NT;
    const int le = t / NT, r = t - le * NT;
    const int a = r / N1, c = r - (r / N1) * N1;
    const int e = blockIdx.x * epb + le;
    const bool valid = e < ne;
    double *T = smem + 6 * NT + le * NA;
    const int nf = in1 ? 2 : 1;
    __syncthreads();
    for (int f = 0; f < nf; ++f) {
        const double *in = f ? in1 : in0;
        double *out = f ? out1 : out0;
        double x[N1], y[N1];
        // (1) x: thread = line (k = a, j = c)
        if (valid) {
            const size_t row = ((size_t)e * NT + a * N1 + c) * N1;
#pragma unroll
            for (int i = 0; i < N1; ++i) x[i] = in[row + i];
#pragma unroll
            for (int q = 0; q < N1; ++q) {
                double s = 0;
#pragma unroll
                for (int i = 0; i < N1; ++i) s += sM[q * N1 + i] * x[i];
                T[(a * N1 + c) * N1 + q] = s;
            }
        }
        __syncthreads();
        // (2) y: thread = (k = a, i = c), column over j
        if (valid) {
#pragma unroll
            for (int j = 0; j < N1; ++j) x[j] = T[(a * N1 + j) * N1 + c];
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                double s = 0;
#pragma unroll
                for (int j = 0; j < N1; ++j) s += sM[NT + m * N1 + j] * x[j];
                T[(a * N1 + m) * N1 + c] = s;
            }
        }
        __syncthreads();
        // (3) z: thread = (j = a, i = c), column over k; then D
        if (valid) {
#pragma unroll
            for (int k = 0; k < N1; ++k) x[k] = T[(k * N1 + a) * N1 + c];
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                double s = 0;
#pragma unroll
                for (int k = 0; k < N1; ++k) s += sM[2 * NT + m * N1 + k] * x[k];
                if (D) s *= D[(m * N1 + a) * N1 + c];
                y[m] = s;
            }
        }
        if (!Cx) {
            if (valid) {
#pragma unroll
                for (int m = 0; m < N1; ++m) out[((size_t)e * NT + m * N1 + a) * N1 + c] = y[m];
            }
            __syncthreads();
            continue;
        }
        // (4) Cz along z (same thread layout), back into the thread's own column of the tile
        if (valid) {
#pragma unroll
            for (int r2 = 0; r2 < N1; ++r2) {
                double s = 0;
#pragma unroll
                for (int m = 0; m < N1; ++m) s += sM[5 * NT + r2 * N1 + m] * y[m];
                T[(r2 * N1 + a) * N1 + c] = s;
            }
        }
        __syncthreads();
        // (5) Cy along y: thread = (k = a, i = c)
        if (valid) {
#pragma unroll
            for (int j = 0; j < N1; ++j) x[j] = T[(a * N1 + j) * N1 + c];
#pragma unroll
            for (int m = 0; m < N1; ++m) {
                double s = 0;
#pragma unroll
                for (int j = 0; j < N1; ++j) s += sM[4 * NT + m * N1 + j] * x[j];
                T[(a * N1 + m) * N1 + c] = s;
            }
        }
        __syncthreads();
        // (6) Cx along x: thread = line (k = a, j = c)
        if (valid) {
            const size_t row = ((size_t)e * NT + a * N1 + c) * N1;
#pragma unroll
            for (int i = 0; i < N1; ++i) x[i] = T[(a * N1 + c) * N1 + i];
#pragma unroll
            for (int q = 0; q < N1; ++q) {
                double s = 0;
#pragma unroll
                for (int i = 0; i < N1; ++i) s += sM[3 * NT + q * N1 + i] * x[i];
                out[row + q] = s;
            }
        }
        __syncthreads();
    }
}

// energy partials: sum over modes of (|Vbar|^2 - lam2 Ubar^2), lam2 = -c2 lambda
template <int N1>
__global__ void k_energy_partial3(int ne, const double *yU, const double *yV, const double *lam2, double *partial) {
    __shared__ double red[1024];
    const int t = threadIdx.x;
    constexpr int ents = N1 * N1 * N1;
    double s = 0.0;
    const long long total = (long long)ne * ents;
    for (long long i = (long long)blockIdx.x * blockDim.x + t; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i % ents);
        const double u = yU[i], v = yV[i];
        s += v * v - lam2[m] * u * u;
    }
    red[t] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) partial[blockIdx.x] = red[0];
}

#define GDG_N1_CASES3(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

int epb3(int n1) { return std::max(1, MAXB3 / (n1 * n1)); }
// per element the fluxes and the tile; per block the parity kernel's c^2 eL / 2 table
size_t smem_stage3(int n1) { return ((size_t)epb3(n1) * (12 * n1 * n1 + 2 * n1 * n1 * n1) + 3 * n1) * sizeof(double); }
size_t smem_traces3(int n1) { return (size_t)epb3(n1) * 2 * n1 * n1 * n1 * sizeof(double); }
size_t smem_sep3(int n1) { return (size_t)(6 * n1 * n1 + epb3(n1) * n1 * n1 * n1) * sizeof(double); }

template <int N1>
void launch_stage3(int mode, const ModalParams &mp, const StageBufs &b, double cA, double cY, cudaStream_t s) {
    const int epb = epb3(N1);
    const dim3 grid((mp.ne + epb - 1) / epb), block(epb * N1 * N1);
    const size_t sm = smem_stage3(N1);
    if (mp.parity) {
        switch (mode) {
#define GDG_K3P(m) (mp.alt ? k_stage3p<N1, m, 1> : k_stage3p<N1, m, 0>)
        case M_RHS: GDG_K3P(M_RHS)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
        case M_S1: GDG_K3P(M_S1)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
        case M_S23: GDG_K3P(M_S23)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
        default: GDG_K3P(M_S4)<<<grid, block, sm, s>>>(mp, b, cA, cY); break;
#undef GDG_K3P
        }
        return;
    }
    switch (mode) {
    case M_RHS: k_stage3<N1, M_RHS><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    case M_S1: k_stage3<N1, M_S1><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    case M_S23: k_stage3<N1, M_S23><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    default: k_stage3<N1, M_S4><<<grid, block, sm, s>>>(mp, b, cA, cY); break;
    }
}

}  // namespace

void gdg3_stage(const ModalParams &mp, int n1, int mode, const StageBufs &b, double cA, double cY, cudaStream_t s) {
    switch (n1) {
#define X(n) case n: launch_stage3<n>(mode, mp, b, cA, cY, s); break;
        GDG_N1_CASES3(X)
#undef X
    }
}

void gdg3_traces(const ModalParams &mp, int n1, const double *yU, const double *yV, double *tr, cudaStream_t s) {
    const int epb = epb3(n1);
    const dim3 grid((mp.ne + epb - 1) / epb), block(epb * n1 * n1);
    switch (n1) {
#define X(n) case n: k_traces3<n><<<grid, block, smem_traces3(n), s>>>(mp, yU, yV, tr); break;
        GDG_N1_CASES3(X)
#undef X
    }
}

void gdg3_sep(int n1, int ne, const double *in0, const double *in1, double *out0, double *out1, const double *Bx,
              const double *By, const double *Bz, const double *D, const double *Cx, const double *Cy,
              const double *Cz, cudaStream_t s) {
    const int epb = epb3(n1);
    const dim3 grid((ne + epb - 1) / epb), block(epb * n1 * n1);
    switch (n1) {
#define X(n) case n: k_sep3<n><<<grid, block, smem_sep3(n), s>>>(ne, in0, in1, out0, out1, Bx, By, Bz, D, Cx, Cy, Cz); break;
        GDG_N1_CASES3(X)
#undef X
    }
}

void gdg3_energy_partial(int n1, int ne, const double *yU, const double *yV, const double *lam2, double *partial,
                         int blocks, cudaStream_t s) {
    switch (n1) {
#define X(n) case n: k_energy_partial3<n><<<blocks, 256, 0, s>>>(ne, yU, yV, lam2, partial); break;
        GDG_N1_CASES3(X)
#undef X
    }
}

void gdg3_set_smem_limits() {
    const int lim = 200 * 1024;
#define X(n)                                                                                    \
    cudaFuncSetAttribute(k_stage3<n, M_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage3<n, M_S1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage3<n, M_S23>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage3<n, M_S4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage3p<n, M_RHS, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage3p<n, M_S1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage3p<n, M_S23, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage3p<n, M_S4, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage3p<n, M_RHS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage3p<n, M_S1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_stage3p<n, M_S23, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
    cudaFuncSetAttribute(k_stage3p<n, M_S4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);  \
    cudaFuncSetAttribute(k_traces3<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);       \
    cudaFuncSetAttribute(k_sep3<n>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    GDG_N1_CASES3(X)
#undef X
}

// this translation unit's check slot (gdg_checks.cuh)
GDG_CHECKS_READER(gdg_checks_read_const3)
