// Variable-coefficient / mapped-element path of libgdg (Section 7.1).
//
// For a variable speed of sound or a non-Cartesian element the simultaneous
// diagonalisation does not apply; the method keeps the nodal GD basis and
// inverts the element matrices of Eqs. DG1 / DG2 by preconditioned CG.
// Geometry (x, y) and c^2 are given at every element's GD nodes and
// represented in the element's own GD space; integrals use nq Gauss points
// per GD cell per direction (Q = N*nq points per direction):
//   M_J  = int phi_a phi_b |J|,   S_c2 = int c^2 grad phi_a . grad phi_b |J|
//   r_u  = sum_faces int_face c^2 (n.grad phi) (v* - v_in) dS
//   r_v  = -S_c2 U + sum_faces int_face c^2 phi q* dS
//   (S_c2 + w w^T) y = r_u, w = M_J 1 / |e|, |e| = 1^T M_J 1 (SPD form of Eq. DG1
//   with DG1_extra; the 1/|e| weight keeps the rank-one term O(1))
//   M_J dV/dt = r_v,  dU/dt = V + y.
// Preconditioner: the frozen-coefficient modified basis (Section 3.2's
// diagonalisation on the reference element, scaled by the element means of
// the metric c^2 |J| J^-1 J^-T and of |J|), or none.
//
// Kernels (one CTA per element):
//   k_var_geom    quadrature assembly of M_J, S_c2, w and face data
//   k_var_traces  v and n.grad u at the face quadrature points
//   k_var_stage   fluxes + lifts + stiffness + both PCG solves (matrices in
//                 shared memory) + RK combine + traces of the next stage input
//   k_var_pcg     one element PCG (gdg_pcg)
//   k_var_energy  per-element V^T M V + U^T S U
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "gdg_internal.h"

#include "gdg_var_kernels.cuh"

namespace {

// ---------------------------------------------------------- dispatch -----

#define GDG_VAR_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10)

size_t geom_smem(int N1, int Q) {
    const int NA = N1 * N1;
    return sizeof(double) * ((size_t)tab_len(Q, N1) + 3 * NA + 5 * N1 * Q + 4 * Q + 4 * NA + 32);
}
size_t traces_smem(int N1, int Q) { return sizeof(double) * ((size_t)tab_len(Q, N1) + 2 * N1 * N1 + 12 * N1); }

template <int N1>
size_t stage_smem(int Q, bool mixed, bool no_matrix) { return StageSmem<N1>::bytes(Q, mixed, no_matrix); }
size_t invert_smem(int N1) { return sizeof(double) * (2 * (size_t)N1 * N1 * N1 * N1 + (size_t)N1 * N1); }
size_t fold_smem(int N1) { return sizeof(double) * ((size_t)fold_rlen(N1) + 12 * (size_t)N1 + 2 * (size_t)N1 * N1); }

// The dynamic shared-memory limit is a property of the kernel function, shared
// by every context: always raise it to the device's opt-in maximum so that a
// context with smaller needs cannot lower it under another one.
template <int N1>
void set_attrs() {
    int dev = 0, lim = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(k_var_geom<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_traces<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_stage<N1, M_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_stage<N1, M_S1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_stage<N1, M_S23>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_stage<N1, M_S4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_pcg<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_invert<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_var_fold<N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <int N1>
void launch_stage_n(const VarData &D, int mode, const VarBufs &b, double cA, double cY, cudaStream_t s) {
    const dim3 grid(D.vp.ne), block(nthreads_for(N1 * N1));
    const size_t sm = D.smem_stage;
    switch (mode) {
    case M_RHS: k_var_stage<N1, M_RHS><<<grid, block, sm, s>>>(D.vp, b, cA, cY); break;
    case M_S1: k_var_stage<N1, M_S1><<<grid, block, sm, s>>>(D.vp, b, cA, cY); break;
    case M_S23: k_var_stage<N1, M_S23><<<grid, block, sm, s>>>(D.vp, b, cA, cY); break;
    default: k_var_stage<N1, M_S4><<<grid, block, sm, s>>>(D.vp, b, cA, cY); break;
    }
}

void launch_stage_raw(gdg_ctx *ctx, int mode, const VarBufs &b, double cA, double cY, cudaStream_t s) {
    const VarData &D = *ctx->var;
    switch (ctx->n1) {
#define X(n) case n: launch_stage_n<n>(D, mode, b, cA, cY, s); break;
        GDG_VAR_CASES(X)
#undef X
    }
}

// One RK stage.  With an attached network the stage is split in three
// launches: residuals, learned u_t guess, solves from the guess.
void launch_stage(gdg_ctx *ctx, int mode, const VarBufs &b, double cA, double cY, cudaStream_t s) {
    VarData &D = *ctx->var;
    if (!D.learned) {
        GDG_PROF(ctx, GDG_K_PCG, s, launch_stage_raw(ctx, mode, b, cA, cY, s));
        return;
    }
    VarBufs b1 = b;
    b1.part = 1; b1.ru = D.d_ru; b1.rv = D.d_rv;
    GDG_PROF(ctx, GDG_K_RHS, s, launch_stage_raw(ctx, mode, b1, cA, cY, s));
    GDG_PROF(ctx, GDG_K_OTHER, s,
             gdg_mlp_guess_launch(D.d_wbf16, D.d_mlp, D.d_c2feat, D.d_ru, ctx->ne, D.d_x0u, s));
    VarBufs b2 = b;
    b2.part = 2; b2.ru = D.d_ru; b2.rv = D.d_rv; b2.x0u = D.d_x0u;
    GDG_PROF(ctx, GDG_K_PCG, s, launch_stage_raw(ctx, mode, b2, cA, cY, s));
}

void launch_traces_raw(gdg_ctx *ctx, const double *u, const double *v, double *tr, cudaStream_t s) {
    const VarData &D = *ctx->var;
    const dim3 grid(D.vp.ne), block(128);
    switch (ctx->n1) {
#define X(n) case n: k_var_traces<n><<<grid, block, D.smem_traces, s>>>(D.vp, u, v, tr); break;
        GDG_VAR_CASES(X)
#undef X
    }
}

void launch_traces(gdg_ctx *ctx, const double *u, const double *v, double *tr, cudaStream_t s) {
    GDG_PROF(ctx, GDG_K_TRACES, s, launch_traces_raw(ctx, u, v, tr, s));
}

void launch_pcg_raw(gdg_ctx *ctx, int which, const double *b, double *x, cudaStream_t s) {
    const VarData &D = *ctx->var;
    const dim3 grid(ctx->ne), block(nthreads_for(ctx->n1 * ctx->n1));
    switch (ctx->n1) {
#define X(n) case n: k_var_pcg<n><<<grid, block, D.smem_pcg, s>>>(D.vp, which == GDG_OP_S, b, x, D.d_iters, D.d_rel, D.d_sweeps); break;
        GDG_VAR_CASES(X)
#undef X
    }
}

double *vbuf(gdg_ctx *ctx, int i) { return ctx->var->d_state + (size_t)i * ctx->ndof; }
enum { B_NU = 0, B_NV, B_AU, B_AV, B_XU, B_XV, B_YU, B_YV, B_COUNT };

void enqueue_step(gdg_ctx *ctx, double dt, cudaStream_t s) {
    VarData &D = *ctx->var;
    double *tr0 = D.d_tr, *tr1 = D.d_tr + D.tr_len;
    VarBufs b{};
    b.nU = vbuf(ctx, B_NU); b.nV = vbuf(ctx, B_NV);
    b.aU = vbuf(ctx, B_AU); b.aV = vbuf(ctx, B_AV);
    b.yU = b.nU; b.yV = b.nV; b.oU = vbuf(ctx, B_XU); b.oV = vbuf(ctx, B_XV); b.trin = tr0; b.trout = tr1;
    b.tstage = 0.0;
    launch_stage(ctx, M_S1, b, dt / 6.0, 0.5 * dt, s);
    b.yU = vbuf(ctx, B_XU); b.yV = vbuf(ctx, B_XV); b.oU = vbuf(ctx, B_YU); b.oV = vbuf(ctx, B_YV); b.trin = tr1; b.trout = tr0;
    b.tstage = 0.5 * dt;
    launch_stage(ctx, M_S23, b, dt / 3.0, 0.5 * dt, s);
    b.yU = vbuf(ctx, B_YU); b.yV = vbuf(ctx, B_YV); b.oU = vbuf(ctx, B_XU); b.oV = vbuf(ctx, B_XV); b.trin = tr0; b.trout = tr1;
    b.tstage = 0.5 * dt;
    launch_stage(ctx, M_S23, b, dt / 3.0, dt, s);
    b.yU = vbuf(ctx, B_XU); b.yV = vbuf(ctx, B_XV); b.oU = nullptr; b.oV = nullptr; b.trin = tr1; b.trout = tr0;
    b.tstage = dt;   // the source block also advances the source time by dt
    launch_stage(ctx, M_S4, b, dt / 6.0, 0.0, s);
}

int check_stats_noconv(gdg_ctx *ctx, cudaStream_t s, int *unconv) {
    unsigned long long h[7];
    int st = gdg_cuda_check(ctx, cudaMemcpyAsync(h, ctx->var->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s), "stats");
    if (!st) st = gdg_cuda_check(ctx, cudaStreamSynchronize(s), "stats sync");
    if (st) return st;
    *unconv = (int)(h[4] + h[5]);
    return GDG_OK;
}

}  // namespace

// --------------------------------------------------------------- API -----

int gdg_var_setup(gdg_ctx *ctx) {
    if (ctx->n1 > GDG_VAR_MAXN1)
        return gdg_set_err(ctx, GDG_EUNSUPPORTED, "variable coefficients need N+1 <= 10");
    VarData *D = new (std::nothrow) VarData();
    if (!D) return GDG_ENOMEM;
    ctx->var = D;
    const int n1 = ctx->n1, NA = n1 * n1, N = ctx->N, p = ctx->p;
    D->nq = ctx->pb.nquad > 0 ? ctx->pb.nquad : p + 1;
    D->Q = N * D->nq;
    D->NA = NA;
    const int Q = D->Q;
    // 1-D tables on the host: composite Gauss rule, basis values / slopes at the points
    std::vector<double> gx, gw;
    gdg_gauss_legendre(D->nq, gx, gw);
    std::vector<double> tab(tab_len(Q, n1), 0.0);
    double *B = tab.data(), *Dd = B + Q * n1, *wq = Dd + Q * n1, *dL = wq + Q, *dR = dL + n1, *Ps = dR + n1,
           *lam = Ps + n1 * n1;
    for (int k = 0; k < N; ++k)
        for (int g = 0; g < D->nq; ++g) {
            const int q = k * D->nq + g;
            gdg_eval_basis(p, N, (k + gx[g]) / N, k, B + q * n1, Dd + q * n1);
            wq[q] = gw[g] / N;
        }
    for (int i = 0; i < n1; ++i) { dL[i] = ctx->dphiL[i]; dR[i] = ctx->dphiR[i]; lam[i] = ctx->lamh[i]; }
    for (int i = 0; i < NA; ++i) Ps[i] = ctx->Psih[i];
    // modes in parity order (the even ones first, each class in the original
    // ascending-lambda order, so the constant mode stays first) where the
    // basis has the r -> 1-r symmetry: the FP64 preconditioner then works by
    // node pairs (precondition_parity)
    bool parity = true;
    {
        double big = 0.0;
        for (int i = 0; i < NA; ++i) big = std::max(big, std::fabs(Ps[i]));
        std::vector<int> ev, od;
        for (int k = 0; k < n1 && parity; ++k) {
            bool even = true, odd = true;
            for (int i = 0; i < n1; ++i) {
                const double a = Ps[i * n1 + k], m = Ps[(n1 - 1 - i) * n1 + k];
                if (std::fabs(m - a) > 1e-9 * big) even = false;
                if (std::fabs(m + a) > 1e-9 * big) odd = false;
            }
            if (even) ev.push_back(k);
            else if (odd) od.push_back(k);
            else parity = false;
        }
        parity = parity && (int)ev.size() == (n1 + 1) / 2 && ev[0] == 0;
        if (parity) {
            std::vector<int> order(ev);
            order.insert(order.end(), od.begin(), od.end());
            const std::vector<double> P0(Ps, Ps + NA), L0(lam, lam + n1);
            for (int k = 0; k < n1; ++k) {
                lam[k] = L0[order[k]];
                for (int i = 0; i < n1; ++i) Ps[i * n1 + k] = P0[i * n1 + order[k]];
            }
        }
    }

    const size_t nd = (size_t)ctx->ndof;
    int st;
    D->tr_len = (long long)ctx->ne * 12 * n1;   // face lines: 4 faces x 3 N1 per element
    if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_S, nd * NA * sizeof(double)), "alloc S")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_M, nd * NA * sizeof(double)), "alloc M")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_w, nd * sizeof(double)), "alloc w")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_pre, (size_t)ctx->ne * 4 * sizeof(double)), "alloc pre")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_face, (size_t)ctx->ne * 16 * Q * sizeof(double)), "alloc face")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_tab, tab.size() * sizeof(double)), "alloc tab")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_nodes, 3 * nd * sizeof(double)), "alloc nodes")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_state, (size_t)B_COUNT * nd * sizeof(double)), "alloc state")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_tr, 2 * (size_t)D->tr_len * sizeof(double)), "alloc tr")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_stats, 16 * sizeof(unsigned long long)), "alloc stats")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_sweeps, (size_t)ctx->ne * sizeof(int)), "alloc sweeps")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_iters, (size_t)ctx->ne * sizeof(int)), "alloc iters")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_rel, (size_t)ctx->ne * sizeof(double)), "alloc rel")) ||
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_red, ((size_t)ctx->ne + 1) * sizeof(double)), "alloc red")) ||
        (st = gdg_cuda_check(ctx, cudaMallocHost((void **)&D->h_red, 8 * sizeof(double)), "alloc host")))
        return st;
    cudaMemset(D->d_stats, 0, 16 * sizeof(unsigned long long));
    cudaMemset(D->d_sweeps, 0, (size_t)ctx->ne * sizeof(int));
    if ((st = gdg_cuda_check(ctx, cudaMemcpy(D->d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice), "upload")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpy(D->d_nodes, ctx->pb.x_nodes, nd * sizeof(double), cudaMemcpyHostToDevice), "upload x")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpy(D->d_nodes + nd, ctx->pb.y_nodes, nd * sizeof(double), cudaMemcpyHostToDevice), "upload y")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpy(D->d_nodes + 2 * nd, ctx->pb.c2_nodes, nd * sizeof(double), cudaMemcpyHostToDevice), "upload c2")))
        return st;
    {   // parallelogram elements: nodes an affine function of the (equispaced) reference nodes
        const double *Xh = ctx->pb.x_nodes, *Yh = ctx->pb.y_nodes;
        std::vector<unsigned char> aff((size_t)ctx->ne, 0);
        for (int e = 0; e < ctx->ne; ++e) {
            const double *x = Xh + (size_t)e * NA, *y = Yh + (size_t)e * NA;
            const double ax = x[1] - x[0], bx = x[n1] - x[0], ay = y[1] - y[0], by = y[n1] - y[0];
            const double tol = 1e-12 * (std::fabs(ax) + std::fabs(bx) + std::fabs(ay) + std::fabs(by));
            bool ok = true;
            for (int j = 0; j < n1 && ok; ++j)
                for (int i = 0; i < n1 && ok; ++i)
                    ok = std::fabs(x[j * n1 + i] - (x[0] + i * ax + j * bx)) <= tol &&
                         std::fabs(y[j * n1 + i] - (y[0] + i * ay + j * by)) <= tol;
            aff[e] = ok;
        }
        if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_affine, aff.size()), "alloc affine")) ||
            (st = gdg_cuda_check(ctx, cudaMemcpy(D->d_affine, aff.data(), aff.size(), cudaMemcpyHostToDevice),
                                 "upload affine")))
            return st;
    }
    VarParams &P = D->vp;
    P.nx = ctx->nx; P.ny = ctx->ny; P.ne = ctx->ne; P.Q = Q;
    P.affine = D->d_affine;
    P.parity = parity;
    P.per_x = ctx->pb.bc[0] == GDG_BC_PERIODIC;
    P.per_y = ctx->pb.bc[1] == GDG_BC_PERIODIC;
    P.upwind = ctx->pb.flux == GDG_FLUX_UPWIND;
    P.alt = ctx->pb.flux == GDG_FLUX_ALTERNATING;
    P.xi = ctx->pb.xi;
    P.rtol = ctx->pb.pcg_rtol;
    P.maxit = ctx->pb.pcg_maxit;
    P.precond = ctx->pb.precond;
    P.tab = D->d_tab; P.S = D->d_S; P.M = D->d_M; P.w = D->d_w; P.pre = D->d_pre; P.face = D->d_face;
    P.stats = D->d_stats;
    P.mixed = ctx->pb.precision == GDG_MIXED;
    P.refine_max = ctx->pb.refine_max > 0 ? ctx->pb.refine_max : 8;
    P.refine_rtol = (float)(ctx->pb.refine_rtol > 0.0 ? ctx->pb.refine_rtol : 1e-5);
    D->smem_geom = geom_smem(n1, Q);
    D->smem_traces = traces_smem(n1, Q);
    switch (n1) {
#define X(n)                                                                                   \
    case n:                                                                                    \
        D->smem_stage = stage_smem<n>(Q, ctx->pb.precision == GDG_MIXED, ctx->pb.solver == GDG_SOLVE_INVERSE); \
        D->smem_pcg = stage_smem<n>(Q, ctx->pb.precision == GDG_MIXED, false);                  \
        set_attrs<n>();                                                                        \
        break;
        GDG_VAR_CASES(X)
#undef X
    }
    if (D->smem_pcg > 220 * 1024 || D->smem_geom > 220 * 1024 ||
        (ctx->pb.solver == GDG_SOLVE_INVERSE && (invert_smem(n1) > 220 * 1024 || fold_smem(n1) > 220 * 1024)))
        return gdg_set_err(ctx, GDG_EUNSUPPORTED, "element too large for shared memory (reduce nquad)");
    const double *Xd = D->d_nodes, *Yd = D->d_nodes + nd, *Cd = D->d_nodes + 2 * nd;
    switch (n1) {
#define X(n) case n: k_var_geom<n><<<ctx->ne, GEOM_THREADS, D->smem_geom>>>(P, Xd, Yd, Cd, D->d_S, D->d_M, D->d_w, D->d_pre, D->d_face); break;
        GDG_VAR_CASES(X)
#undef X
    }
    // face operators: 4 faces x 6 N1 columns x 3 N1 rows per element, from the face data
    if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_FM, (size_t)ctx->ne * 72 * n1 * n1 * sizeof(double)), "alloc FM")))
        return st;
    switch (n1) {
#define X(n) case n: k_var_facemat<n><<<ctx->ne, nthreads_for(n * n), 3 * (size_t)Q * sizeof(double)>>>(P, D->d_FM); break;
        GDG_VAR_CASES(X)
#undef X
    }
    P.FM = D->d_FM;
    P.src_e = -1;   // no point source until gdg_set_point_source
    if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_time, sizeof(double)), "alloc time")) ||
        (st = gdg_cuda_check(ctx, cudaMemset(D->d_time, 0, sizeof(double)), "time")))
        return st;
    P.time = D->d_time;
    {   // c^2 / element mean of c^2 at the nodes: features of the learned u_t guess
        std::vector<float> feat(nd);
        for (int e = 0; e < ctx->ne; ++e) {
            double m = 0.0;
            for (int a = 0; a < NA; ++a) m += ctx->pb.c2_nodes[(size_t)e * NA + a];
            m /= NA;
            for (int a = 0; a < NA; ++a) feat[(size_t)e * NA + a] = (float)(ctx->pb.c2_nodes[(size_t)e * NA + a] / m);
        }
        if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_c2feat, nd * sizeof(float)), "alloc features")) ||
            (st = gdg_cuda_check(ctx, cudaMemcpy(D->d_c2feat, feat.data(), nd * sizeof(float), cudaMemcpyHostToDevice), "upload features")))
            return st;
    }
    if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_dS, nd * sizeof(double)), "alloc dS"))) return st;
    switch (n1) {
#define X(n) case n: k_fdm_diag<n><<<ctx->ne, nthreads_for(n * n)>>>(D->d_tab + tab_len(Q, n) - n, D->d_pre, D->d_dS); break;
        GDG_VAR_CASES(X)
#undef X
    }
    P.dS = D->d_dS;
    P.inverse = ctx->pb.solver == GDG_SOLVE_INVERSE;
    if (P.inverse) {   // element inverses (S_c2 + w w^T)^-1 and M_J^-1, folded with the lifts
        const size_t nm = nd * NA;
        if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_Ainv, nm * sizeof(double)), "alloc Ainv")) ||
            (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_Minv, nm * sizeof(double)), "alloc Minv")) ||
            (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_G, nd * fold_cols(n1) * sizeof(double)), "alloc G")))
            return st;
        const size_t ism = invert_smem(n1), fsm = fold_smem(n1);
        switch (n1) {
#define X(n)                                                                                         \
    case n:                                                                                          \
        k_var_invert<n><<<ctx->ne, nthreads_for(n * n), ism>>>(D->d_S, D->d_w, D->d_Ainv);           \
        k_var_invert<n><<<ctx->ne, nthreads_for(n * n), ism>>>(D->d_M, nullptr, D->d_Minv);          \
        k_var_fold<n><<<ctx->ne, nthreads_for(n * n), fsm>>>(D->d_S, D->d_Ainv, D->d_Minv, D->d_tab, Q, D->d_G); \
        break;
            GDG_VAR_CASES(X)
#undef X
        }
        P.G = D->d_G;
    }
    if (P.mixed) {   // FP32 copies of the element matrices (packed lower triangles) for the inner solves
        const size_t nm = (size_t)ctx->ne * tri_len(NA);
        if ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_S32, nm * sizeof(float)), "alloc S32")) ||
            (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D->d_M32, nm * sizeof(float)), "alloc M32")))
            return st;
        const int grid = (int)std::min<long long>(ctx->ne, 65535);
        switch (n1) {
#define X(n)                                                                  \
    case n:                                                                   \
        k_to_f32_lower<n><<<grid, 128>>>(ctx->ne, D->d_S, D->d_S32);          \
        k_to_f32_lower<n><<<grid, 128>>>(ctx->ne, D->d_M, D->d_M32);          \
        break;
            GDG_VAR_CASES(X)
#undef X
        }
        P.S32 = D->d_S32;
        P.M32 = D->d_M32;
    }
    st = gdg_cuda_check(ctx, cudaDeviceSynchronize(), "assembly");
    cudaFree(D->d_nodes);
    cudaFree(D->d_Ainv);
    cudaFree(D->d_Minv);
    D->d_nodes = D->d_Ainv = D->d_Minv = nullptr;
    if (st) return st;
    // the mapping must be orientation preserving: every frozen |J| mean > 0
    std::vector<double> pre((size_t)ctx->ne * 4);
    cudaMemcpy(pre.data(), D->d_pre, pre.size() * sizeof(double), cudaMemcpyDeviceToHost);
    for (int e = 0; e < ctx->ne; ++e)
        if (!(pre[(size_t)e * 4 + 2] > 0.0) || !std::isfinite(pre[(size_t)e * 4 + 0]))
            return gdg_set_err(ctx, GDG_EINVAL, "element mapping is degenerate or not orientation preserving");
    return gdg_cuda_check(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "stream");
}

void gdg_var_free(gdg_ctx *ctx) {
    VarData *D = ctx->var;
    if (!D) return;
    cudaFree(D->d_S); cudaFree(D->d_M); cudaFree(D->d_S32); cudaFree(D->d_M32); cudaFree(D->d_dS); cudaFree(D->d_Ainv); cudaFree(D->d_Minv); cudaFree(D->d_G); cudaFree(D->d_FM); cudaFree(D->d_time); cudaFree(D->d_src); cudaFree(D->d_w); cudaFree(D->d_pre); cudaFree(D->d_face); cudaFree(D->d_affine);
    cudaFree(D->d_tab); cudaFree(D->d_nodes); cudaFree(D->d_state); cudaFree(D->d_tr);
    cudaFree(D->d_c2feat); cudaFree(D->d_wbf16); cudaFree(D->d_mlp);
    cudaFree(D->d_ru); cudaFree(D->d_rv); cudaFree(D->d_x0u);
    cudaFree(D->d_stats); cudaFree(D->d_iters); cudaFree(D->d_sweeps); cudaFree(D->d_rel); cudaFree(D->d_red);
    if (D->h_red) cudaFreeHost(D->h_red);
    delete D;
    ctx->var = nullptr;
}

int gdg_var_rhs(gdg_ctx *ctx, const double *u, const double *v, double t, double *du, double *dv,
                cudaStream_t s) {
    VarData &D = *ctx->var;
    if (D.vp.src_e >= 0) k_set_time<<<1, 1, 0, s>>>(D.d_time, t);   // the forcing's time
    cudaMemsetAsync(D.d_stats, 0, 16 * sizeof(unsigned long long), s);
    launch_traces(ctx, u, v, D.d_tr, s);
    VarBufs b{};
    b.yU = u; b.yV = v; b.oU = du; b.oV = dv; b.trin = D.d_tr;
    launch_stage(ctx, M_RHS, b, 0.0, 0.0, s);
    int st = gdg_cuda_check(ctx, cudaGetLastError(), "gdg_rhs launch");
    if (st) return st;
    int unconv = 0;
    if ((st = check_stats_noconv(ctx, s, &unconv))) return st;
    return unconv ? gdg_set_err(ctx, GDG_ENOCONV, "PCG hit pcg_maxit") : GDG_OK;
}

int gdg_var_pcg(gdg_ctx *ctx, int which, const double *b, double *x, gdg_pcg_stats *stats, cudaStream_t s) {
    VarData &D = *ctx->var;
    GDG_PROF(ctx, GDG_K_PCG, s, launch_pcg_raw(ctx, which, b, x, s));
    int st = gdg_cuda_check(ctx, cudaGetLastError(), "gdg_pcg launch");
    if (st || !stats) return st;
    std::vector<int> it(ctx->ne), sw(ctx->ne);
    std::vector<double> rel(ctx->ne);
    if ((st = gdg_cuda_check(ctx, cudaMemcpyAsync(it.data(), D.d_iters, it.size() * sizeof(int), cudaMemcpyDeviceToHost, s), "iters")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpyAsync(sw.data(), D.d_sweeps, sw.size() * sizeof(int), cudaMemcpyDeviceToHost, s), "sweeps")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpyAsync(rel.data(), D.d_rel, rel.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "rel")) ||
        (st = gdg_cuda_check(ctx, cudaStreamSynchronize(s), "pcg sync")))
        return st;
    stats->max_iters = 0;
    stats->mean_iters = 0.0;
    stats->max_rel_resid = 0.0;
    stats->unconverged = 0;
    stats->max_sweeps = 0;
    stats->mean_sweeps = 0.0;
    stats->guessed = 0;
    stats->fell_back = 0;
    bool nonfinite = false;
    const bool mixed = ctx->pb.precision == GDG_MIXED;
    for (int e = 0; e < ctx->ne; ++e) {
        stats->max_iters = it[e] > stats->max_iters ? it[e] : stats->max_iters;
        stats->mean_iters += it[e];
        if (mixed) {
            stats->max_sweeps = sw[e] > stats->max_sweeps ? sw[e] : stats->max_sweeps;
            stats->mean_sweeps += sw[e];
        }
        if (!std::isfinite(rel[e])) nonfinite = true;
        else if (rel[e] > stats->max_rel_resid) stats->max_rel_resid = rel[e];
        const bool capped = mixed ? sw[e] >= ctx->pb.refine_max : it[e] >= ctx->pb.pcg_maxit;
        if (capped && rel[e] > ctx->pb.pcg_rtol) stats->unconverged++;
    }
    stats->mean_iters /= ctx->ne;
    stats->mean_sweeps /= ctx->ne;
    if (nonfinite) return gdg_set_err(ctx, GDG_ENONFINITE, "non-finite PCG residual");
    if (stats->unconverged) return gdg_set_err(ctx, GDG_ENOCONV, "PCG hit pcg_maxit");
    return GDG_OK;
}

int gdg_var_step(gdg_ctx *ctx, double *u, double *v, double t0, double dt, int nsteps, cudaStream_t s) {
    VarData &D = *ctx->var;
    const size_t bytes = (size_t)ctx->ndof * sizeof(double);
    int st;
    if (D.vp.src_e >= 0) k_set_time<<<1, 1, 0, s>>>(D.d_time, t0);
    if ((st = gdg_cuda_check(ctx, cudaMemcpyAsync(vbuf(ctx, B_NU), u, bytes, cudaMemcpyDeviceToDevice, s), "copy u")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpyAsync(vbuf(ctx, B_NV), v, bytes, cudaMemcpyDeviceToDevice, s), "copy v")))
        return st;
    launch_traces(ctx, vbuf(ctx, B_NU), vbuf(ctx, B_NV), D.d_tr, s);
    const int G = (nsteps >= 8 && !ctx->prof.on) ? 8 : 0;
    if (G) {
        GraphCache &gc = ctx->graph;
        if (!gc.exec || gc.dt != dt || gc.steps != G) {
            if (gc.exec) cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
            cudaGraph_t g;
            if ((st = gdg_cuda_check(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal), "capture")))
                return st;
            for (int i = 0; i < G; ++i) enqueue_step(ctx, dt, ctx->cap_stream);
            if ((st = gdg_cuda_check(ctx, cudaStreamEndCapture(ctx->cap_stream, &g), "capture end"))) return st;
            st = gdg_cuda_check(ctx, cudaGraphInstantiate(&gc.exec, g, 0), "instantiate");
            cudaGraphDestroy(g);
            if (st) return st;
            gc.dt = dt;
            gc.steps = G;
        }
        for (int i = 0; i + G <= nsteps; i += G)
            if ((st = gdg_cuda_check(ctx, cudaGraphLaunch(gc.exec, s), "graph launch"))) return st;
    }
    const int rem = G ? nsteps % G : nsteps;
    for (int i = 0; i < rem; ++i) enqueue_step(ctx, dt, s);
    if ((st = gdg_cuda_check(ctx, cudaMemcpyAsync(u, vbuf(ctx, B_NU), bytes, cudaMemcpyDeviceToDevice, s), "copy u")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpyAsync(v, vbuf(ctx, B_NV), bytes, cudaMemcpyDeviceToDevice, s), "copy v")))
        return st;
    return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_step");
}

int gdg_var_energy(gdg_ctx *ctx, const double *u, const double *v, double *E, cudaStream_t s) {
    VarData &D = *ctx->var;
    const dim3 grid(ctx->ne), block(nthreads_for(ctx->n1 * ctx->n1));
    switch (ctx->n1) {
#define X(n) case n: k_var_energy<n><<<grid, block, 0, s>>>(D.vp, u, v, D.d_red); break;
        GDG_VAR_CASES(X)
#undef X
    }
    k_var_sum<<<1, 1024, 0, s>>>(ctx->ne, D.d_red, D.d_red + ctx->ne);
    int st;
    if ((st = gdg_cuda_check(ctx, cudaMemcpyAsync(D.h_red, D.d_red + ctx->ne, sizeof(double), cudaMemcpyDeviceToHost, s), "energy d2h")) ||
        (st = gdg_cuda_check(ctx, cudaStreamSynchronize(s), "energy sync")))
        return st;
    *E = D.h_red[0];
    return GDG_OK;
}

int gdg_var_step_stats(gdg_ctx *ctx, gdg_pcg_stats *su, gdg_pcg_stats *sv) {
    unsigned long long h[16];
    int st = gdg_cuda_check(ctx, cudaMemcpy(h, ctx->var->d_stats, sizeof(h), cudaMemcpyDeviceToHost), "stats");
    if (st) return st;
    const double n = h[6] ? (double)h[6] : 1.0;
    if (su) {
        su->max_iters = (int)h[2]; su->mean_iters = h[0] / n; su->max_rel_resid = 0.0; su->unconverged = (int)h[4];
        su->max_sweeps = (int)h[9]; su->mean_sweeps = h[7] / n;
        su->guessed = (long long)h[11]; su->fell_back = (long long)h[12];
    }
    if (sv) {
        sv->max_iters = (int)h[3]; sv->mean_iters = h[1] / n; sv->max_rel_resid = 0.0; sv->unconverged = (int)h[5];
        sv->max_sweeps = (int)h[10]; sv->mean_sweeps = h[8] / n;
        sv->guessed = 0; sv->fell_back = 0;
    }
    cudaMemset(ctx->var->d_stats, 0, 16 * sizeof(unsigned long long));
    return GDG_OK;
}

StepBuffers gdg_var_buffers(gdg_ctx *ctx) {
    StepBuffers b;
    b.nU = vbuf(ctx, B_NU); b.nV = vbuf(ctx, B_NV); b.aU = vbuf(ctx, B_AU); b.aV = vbuf(ctx, B_AV);
    b.xU = vbuf(ctx, B_XU); b.xV = vbuf(ctx, B_XV); b.yU = vbuf(ctx, B_YU); b.yV = vbuf(ctx, B_YV);
    b.tr0 = ctx->var->d_tr; b.tr1 = ctx->var->d_tr + ctx->var->tr_len;
    return b;
}

int gdg_var_enter(gdg_ctx *ctx, const double *u, const double *v, cudaStream_t s) {
    const size_t bytes = (size_t)ctx->ndof * sizeof(double);
    int st;
    if ((st = gdg_cuda_check(ctx, cudaMemcpyAsync(vbuf(ctx, B_NU), u, bytes, cudaMemcpyDeviceToDevice, s), "copy u")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpyAsync(vbuf(ctx, B_NV), v, bytes, cudaMemcpyDeviceToDevice, s), "copy v")))
        return st;
    launch_traces(ctx, vbuf(ctx, B_NU), vbuf(ctx, B_NV), ctx->var->d_tr, s);
    return gdg_cuda_check(ctx, cudaGetLastError(), "enter");
}

int gdg_var_leave(gdg_ctx *ctx, double *u, double *v, cudaStream_t s) {
    const size_t bytes = (size_t)ctx->ndof * sizeof(double);
    int st;
    if ((st = gdg_cuda_check(ctx, cudaMemcpyAsync(u, vbuf(ctx, B_NU), bytes, cudaMemcpyDeviceToDevice, s), "copy u")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpyAsync(v, vbuf(ctx, B_NV), bytes, cudaMemcpyDeviceToDevice, s), "copy v")))
        return st;
    return GDG_OK;
}

// ------------------------------------------------------- learned guess -----

static int require_var(gdg_ctx *ctx) {
    if (!ctx) return GDG_EINVAL;
    if (!ctx->var) return gdg_set_err(ctx, GDG_EINVAL, "needs a GDG_COEF_NODAL context");
    return GDG_OK;
}

static void drop_graph(gdg_ctx *ctx) {
    if (ctx->graph.exec) cudaGraphExecDestroy(ctx->graph.exec);
    ctx->graph.exec = nullptr;
}

extern "C" int gdg_residuals(gdg_ctx *ctx, const double *u, const double *v, double *ru, double *rv, void *stream) {
    int st = require_var(ctx);
    if (st) return st;
    if (!u || !v || !ru || !rv) return GDG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    launch_traces(ctx, u, v, ctx->var->d_tr, s);
    VarBufs b{};
    b.yU = u; b.yV = v; b.trin = ctx->var->d_tr; b.part = 1; b.ru = ru; b.rv = rv;
    GDG_PROF(ctx, GDG_K_RHS, s, launch_stage_raw(ctx, M_RHS, b, 0.0, 0.0, s));
    return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_residuals");
}

extern "C" int gdg_mlp_rows(gdg_ctx *ctx, const double *ru, const double *y, float *X, float *T, void *stream) {
    int st = require_var(ctx);
    if (st) return st;
    if (!ru || !X || (y && !T)) return GDG_EINVAL;
    gdg_mlp_rows_launch(ctx->var->d_c2feat, ru, y, ctx->ne, X, T, (cudaStream_t)stream);
    return gdg_cuda_check(ctx, cudaGetLastError(), "gdg_mlp_rows");
}

extern "C" int gdg_mlp_attach(gdg_ctx *ctx, const uint16_t *w_bf16, const float *params) {
    int st = require_var(ctx);
    if (st) return st;
    if (!w_bf16 || !params) return GDG_EINVAL;
    if (ctx->pb.solver != GDG_SOLVE_PCG)
        return gdg_set_err(ctx, GDG_EINVAL, "the learned guess needs GDG_SOLVE_PCG");
    VarData &D = *ctx->var;
    const size_t nd = (size_t)ctx->ndof;
    if (!D.d_wbf16 &&
        ((st = gdg_cuda_check(ctx, cudaMalloc((void **)&D.d_wbf16, GDG_MLP_NWEIGHT * sizeof(uint16_t)), "alloc")) ||
         (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D.d_mlp, GDG_MLP_NPARAM * sizeof(float)), "alloc")) ||
         (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D.d_ru, nd * sizeof(double)), "alloc")) ||
         (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D.d_rv, nd * sizeof(double)), "alloc")) ||
         (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D.d_x0u, nd * sizeof(double)), "alloc"))))
        return st;
    if ((st = gdg_cuda_check(ctx, cudaMemcpy(D.d_wbf16, w_bf16, GDG_MLP_NWEIGHT * sizeof(uint16_t), cudaMemcpyDeviceToDevice), "copy")) ||
        (st = gdg_cuda_check(ctx, cudaMemcpy(D.d_mlp, params, GDG_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice), "copy")))
        return st;
    D.learned = 1;
    drop_graph(ctx);
    return GDG_OK;
}

extern "C" int gdg_mlp_detach(gdg_ctx *ctx) {
    int st = require_var(ctx);
    if (st) return st;
    ctx->var->learned = 0;
    drop_graph(ctx);
    return GDG_OK;
}

// ------------------------------------------------------- point source ------

// Point source f(x, t) = amplitude sin(omega t) delta(x - x_s) on the right of
// u_tt = div(c^2 grad u) + f: its load on r_v (int phi_a f) is
// phi_a(x_s) amplitude sin(omega t) on the element holding x_s, with x_s given
// by that element and its reference coordinates (r, s).
extern "C" int gdg_set_point_source(gdg_ctx *ctx, int element, double r, double s, double amplitude,
                                    double omega) {
    int st;
    if ((st = require_var(ctx))) return st;
    if (element < 0 || element >= ctx->ne || !(r >= 0.0 && r <= 1.0) || !(s >= 0.0 && s <= 1.0) ||
        !std::isfinite(amplitude) || !std::isfinite(omega))
        return gdg_set_err(ctx, GDG_EINVAL, "point source: element index, (r, s) in [0,1]^2, finite amplitude and omega");
    VarData &D = *ctx->var;
    // work still running on any stream may read the source buffer and the
    // parameters about to change: wait for it first, as the header states
    if ((st = gdg_cuda_check(ctx, cudaDeviceSynchronize(), "point source: synchronise"))) return st;
    drop_graph(ctx);   // the source is a kernel parameter of the captured launches
    if (amplitude == 0.0) {
        D.vp.src_e = -1;
        return GDG_OK;
    }
    const int n1 = ctx->n1, NA = n1 * n1;
    std::vector<double> pr(n1), dpr(n1), ps(n1), dps(n1), w(2 * (size_t)NA, 0.0);
    gdg_eval_basis(ctx->p, ctx->N, r, -1, pr.data(), dpr.data());
    gdg_eval_basis(ctx->p, ctx->N, s, -1, ps.data(), dps.data());
    for (int j = 0; j < n1; ++j)
        for (int i = 0; i < n1; ++i) w[(size_t)j * n1 + i] = ps[j] * pr[i];
    if (D.vp.inverse) {   // the inverse route adds M_J^-1 w: Gaussian elimination with partial pivoting
        std::vector<double> M((size_t)NA * NA), x(w.begin(), w.begin() + NA);
        if ((st = gdg_cuda_check(ctx, cudaMemcpy(M.data(), D.d_M + (size_t)element * NA * NA, M.size() * sizeof(double),
                                                 cudaMemcpyDeviceToHost), "point source: mass matrix")))
            return st;
        for (int k = 0; k < NA; ++k) {
            int piv = k;
            for (int i = k + 1; i < NA; ++i)
                if (std::fabs(M[(size_t)i * NA + k]) > std::fabs(M[(size_t)piv * NA + k])) piv = i;
            if (piv != k) {
                for (int c = 0; c < NA; ++c) std::swap(M[(size_t)k * NA + c], M[(size_t)piv * NA + c]);
                std::swap(x[k], x[piv]);
            }
            const double d = M[(size_t)k * NA + k];
            if (!(std::fabs(d) > 0.0)) return gdg_set_err(ctx, GDG_EINVAL, "point source: singular mass matrix");
            for (int i = k + 1; i < NA; ++i) {
                const double m = M[(size_t)i * NA + k] / d;
                if (m == 0.0) continue;
                for (int c = k; c < NA; ++c) M[(size_t)i * NA + c] -= m * M[(size_t)k * NA + c];
                x[i] -= m * x[k];
            }
        }
        for (int k = NA - 1; k >= 0; --k) {
            double acc = x[k];
            for (int c = k + 1; c < NA; ++c) acc -= M[(size_t)k * NA + c] * x[c];
            x[k] = acc / M[(size_t)k * NA + k];
        }
        for (int a = 0; a < NA; ++a) w[(size_t)NA + a] = x[a];
    }
    if (!D.d_src && (st = gdg_cuda_check(ctx, cudaMalloc((void **)&D.d_src, 2 * (size_t)NA * sizeof(double)), "alloc source")))
        return st;
    if ((st = gdg_cuda_check(ctx, cudaMemcpy(D.d_src, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice),
                             "point source: upload")))
        return st;
    D.vp.src_e = element;
    D.vp.src_amp = amplitude;
    D.vp.src_omega = omega;
    D.vp.src_w = D.d_src;
    return GDG_OK;
}

// this translation unit's check slot (gdg_checks.cuh)
GDG_CHECKS_READER(gdg_checks_read_var)
