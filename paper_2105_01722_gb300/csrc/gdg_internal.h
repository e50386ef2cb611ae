// Internal declarations shared by the host code and the CUDA translation
// units of libgdg (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "gdg.h"

#define GDG_MAXN1 16

// Per-direction modal operators of the modified GD basis (Section 3.2) in
// physical scaling: Psi^T M Psi = I with M = H * M_hat, lambda = lambda_hat / H^2.
//   eL[k] = Psi[0][k], eR[k] = Psi[N][k]                  (face values)
//   gL[k] = sum_i Psi[i][k] aL[i], gR[k] likewise          (n . grad at faces)
//   aL = -phi'(0)/H (outward -x), aR = phi'(1)/H (outward +x)
struct ModalDir {
    double eL[GDG_MAXN1], eR[GDG_MAXN1], gL[GDG_MAXN1], gR[GDG_MAXN1], lam[GDG_MAXN1];
    // parity kernel: lift vectors with the flux factor 1/2 (and c^2) folded in
    double hgL[GDG_MAXN1], ceL[GDG_MAXN1];
};

// Everything a stage kernel needs besides buffers (passed by value).
struct ModalParams {
    ModalDir d[3];
    int nx, ny, nz, ne;
    int per_x, per_y, per_z;   // periodic flags
    double c2, beta, tau; // fluxes: v* = (vi+vo)/2 - beta(di+do), q* = (di-do)/2 - tau(vi-vo)
    double beta2, tau2;   // 2 beta, 2 tau
    int alt;              // alternating flux (alpha = 1, beta = tau = 0; side 1 = left / lower element)
    int parity;           // modes ordered even (r -> 1-r symmetric) first: eR = +-eL, gR = +-gL
    int epb;              // elements per block of the 2-D kernels
    int epbh;             // elements per block of the half-line stage kernel (2 N1 threads each)
    int split;            // parity stage kernel: 0 one line, 1 half line, 2 field split, 3 persistent step
                          // (chosen by timing)
    int epbp;             // elements per block of the persistent step (0: its grid does not fit)
    int halo_lo, halo_hi; // y sides whose neighbour traces arrive in ghost rows (partitioned mesh)
};

// RK4 stage modes of the stage kernels
enum {
    M_RHS = 0,   // write k = f(Y)
    M_S1 = 1,    // acc = cA k; Y' = Y + cY k         (Y = y_n)
    M_S23 = 2,   // acc += cA k; Y' = y_n + cY k
    M_S4 = 3     // y_n += acc + cA k
};

// Buffers of one modal RK stage launch.
struct StageBufs {
    const double *yU, *yV;   // stage input (modal)
    double *nU, *nV;         // y_n
    double *aU, *aV;         // RK accumulator
    double *oU, *oV;         // next stage input, or k (M_RHS)
    const double *trin;      // traces of the stage input
    double *trout;           // traces of the next stage input
    const double *lam2;      // [2][n1^d] : -c2 * lambda, 1/lambda (0 on mode 0); 2-D: [4][n1^2]
};

// 3-D modal-route launches (gdg_const3.cu), n1 = N+1 in 2..10
void gdg3_stage(const ModalParams &mp, int n1, int mode, const StageBufs &b, double cA, double cY, cudaStream_t s);
void gdg3_traces(const ModalParams &mp, int n1, const double *yU, const double *yV, double *tr, cudaStream_t s);
void gdg3_sep(int n1, int ne, const double *in0, const double *in1, double *out0, double *out1, const double *Bx,
              const double *By, const double *Bz, const double *D, const double *Cx, const double *Cy,
              const double *Cz, cudaStream_t s);
void gdg3_energy_partial(int n1, int ne, const double *yU, const double *yV, const double *lam2, double *partial,
                         int blocks, cudaStream_t s);
void gdg3_set_smem_limits();

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    double dt = 0.0;
    int steps = 0;
    const void *u = nullptr, *v = nullptr;   // nodal-state route: the state the graph steps in place
};

struct VarData;   // variable-coefficient / mapped data (gdg_var.cu)

// CUDA-event bracketing of launches while profiling is enabled
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> recs;
    size_t used = 0;
    cudaEvent_t begin(cudaStream_t s);
    void end(int kind, cudaEvent_t start, cudaStream_t s);
    void clear();
    void destroy();
};

struct gdg_ctx {
    gdg_problem pb{};
    int dim = 1, nx = 1, ny = 1, nz = 1, N = 1, n1 = 2, p = 1, ne = 1;
    long long ndof = 0;      // doubles per field
    int device = 0;
    std::string err;

    // host 1-D reference data
    std::vector<double> Mh, Sh, phiL, phiR, dphiL, dphiR, Psih, lamh;

    // constant-coefficient Cartesian (diagonalised route)
    ModalParams mp{};
    double *d_mats = nullptr;     // device tables: per direction P = Psi^T M, Psi, Psi^T (n1*n1 each)
    double *d_lam2 = nullptr;     // per mode: -c2*lambda, 1/lambda (0 for mode 0); 2-D also P1, P2
                                  // (the u lifts over lambda, see stage2p_body)
    double *d_state = nullptr;    // modal work: yn(2 fields), acc(2), YA(2), YB(2), K(2)
    double *d_tr = nullptr;       // two trace buffers (past the lower ghost row when halo sides exist)
    long long tr_len = 0;         // doubles per trace buffer (ghost rows included)
    double *d_tr_alloc = nullptr; // allocation holding d_tr
    // element-partitioned mesh: caller's exchange buffers and function
    double *halo_send[2] = {nullptr, nullptr}, *halo_recv[2] = {nullptr, nullptr};
    gdg_halo_fn halo_fn = nullptr;
    void *halo_user = nullptr;
    double *d_red = nullptr;      // reduction partials
    int red_len = 0;
    double *h_red = nullptr;      // pinned host scalar(s)
    cudaStream_t cap_stream = nullptr;
    GraphCache graph;
    bool stage_tuned = false;     // stage kernel variant chosen (first gdg_step)
    unsigned *d_sync = nullptr;   // grid barrier of the persistent step: arrivals, give-up flag
    unsigned long long wait_limit_ns = 1000000000ull;   // bound on any device-side wait

    VarData *var = nullptr;
    Profiler prof;
    double *d_io = nullptr;       // device copies for gdg_step_host (2 fields)
};

// bracket one launch when profiling: GDG_PROF(ctx, kind, stream, launch-statement)
#define GDG_PROF(ctx, kind, s, stmt)                                   \
    do {                                                               \
        cudaEvent_t gdg_ev0_ = (ctx)->prof.on ? (ctx)->prof.begin(s) : nullptr; \
        stmt;                                                          \
        if (gdg_ev0_) (ctx)->prof.end((kind), gdg_ev0_, (s));           \
    } while (0)

// error helpers
int gdg_set_err(gdg_ctx *ctx, int status, const std::string &msg);
int gdg_cuda_check(gdg_ctx *ctx, cudaError_t e, const char *where);

// host basis builder (gdg_host.cpp)
int gdg_build_basis(int p, int N, std::vector<double> &M, std::vector<double> &S,
                    std::vector<double> &phiL, std::vector<double> &phiR,
                    std::vector<double> &dphiL, std::vector<double> &dphiR,
                    std::vector<double> &Psi, std::vector<double> &lam);
void gdg_gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
void gdg_eval_basis(int p, int N, double r, int cell, double *phi, double *dphi);

// constant-coefficient path (gdg_const.cu)
int gdg_const_setup(gdg_ctx *ctx);
void gdg_const_free(gdg_ctx *ctx);
int gdg_const_rhs(gdg_ctx *ctx, const double *u, const double *v, double *du, double *dv,
                  cudaStream_t s);
int gdg_const_mass_solve(gdg_ctx *ctx, int which, const double *b, double *x, cudaStream_t s);
int gdg_const_step(gdg_ctx *ctx, double *u, double *v, double dt, int nsteps, cudaStream_t s);
int gdg_const_energy(gdg_ctx *ctx, const double *u, const double *v, double *E, cudaStream_t s);

// variable-coefficient / mapped path (gdg_var.cu)
int gdg_var_setup(gdg_ctx *ctx);
void gdg_var_free(gdg_ctx *ctx);
int gdg_var_rhs(gdg_ctx *ctx, const double *u, const double *v, double t, double *du, double *dv,
                cudaStream_t s);
int gdg_var_pcg(gdg_ctx *ctx, int which, const double *b, double *x, gdg_pcg_stats *st,
                cudaStream_t s);
int gdg_var_step(gdg_ctx *ctx, double *u, double *v, double t0, double dt, int nsteps, cudaStream_t s);
int gdg_var_energy(gdg_ctx *ctx, const double *u, const double *v, double *E, cudaStream_t s);
int gdg_var_step_stats(gdg_ctx *ctx, gdg_pcg_stats *su, gdg_pcg_stats *sv);

// Buffers of one problem's RK4 state as used by the stage kernels (the
// batched launcher drives several problems' stages from one kernel).
struct StepBuffers {
    double *nU, *nV, *aU, *aV, *xU, *xV, *yU, *yV;   // y_n, accumulator, two stage inputs
    double *tr0, *tr1;                               // traces of y_n / odd stages, even stages
};
StepBuffers gdg_const_buffers(gdg_ctx *ctx);
StepBuffers gdg_var_buffers(gdg_ctx *ctx);
// nodal (u, v) -> internal state and its traces; internal state -> nodal
int gdg_const_enter(gdg_ctx *ctx, const double *u, const double *v, cudaStream_t s);
int gdg_const_leave(gdg_ctx *ctx, double *u, double *v, cudaStream_t s);
int gdg_var_enter(gdg_ctx *ctx, const double *u, const double *v, cudaStream_t s);
int gdg_var_leave(gdg_ctx *ctx, double *u, double *v, cudaStream_t s);

// learned-guess kernels (gdg_mlp.cu)
int gdg_mlp_guess_launch(const uint16_t *w_bf16, const float *params, const float *c2feat, const double *ru,
                         int ne, double *x0u, cudaStream_t s);
int gdg_mlp_rows_launch(const float *c2feat, const double *ru, const double *y, int ne, float *X, float *T,
                        cudaStream_t s);
