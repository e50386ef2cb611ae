// Host side of libgdg: the 1-D GD basis builder (Sections 2.1, 2.1.1, 3.1,
// 3.2), problem validation, context life cycle and the C ABI entry points.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "gdg_checks.cuh"
#include "gdg_internal.h"

// --------------------------------------------------------------- errors --

int gdg_set_err(gdg_ctx *ctx, int status, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return status;
}

int gdg_cuda_check(gdg_ctx *ctx, cudaError_t e, const char *where) {
    if (e == cudaSuccess) return GDG_OK;
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return gdg_set_err(ctx, GDG_ENOMEM, m);
    return gdg_set_err(ctx, GDG_ECUDA, m);
}

extern "C" const char *gdg_status_string(int s) {
    switch (s) {
    case GDG_OK: return "ok";
    case GDG_EINVAL: return "invalid argument";
    case GDG_ENOMEM: return "out of memory";
    case GDG_ECUDA: return "CUDA error";
    case GDG_ENOCONV: return "PCG did not converge within pcg_maxit";
    case GDG_ETIMEOUT: return "bounded device wait timed out";
    case GDG_ENONFINITE: return "non-finite value";
    case GDG_EUNSUPPORTED: return "unsupported configuration";
    case GDG_EHALO: return "halo exchange function failed";
    default: return "unknown status";
    }
}

extern "C" const char *gdg_last_error(const gdg_ctx *ctx) {
    return ctx ? ctx->err.c_str() : "";
}

// ---------------------------------------------------- 1-D GD basis -------

// Gauss-Legendre nodes/weights on [0,1]: Newton iteration on P_n with the
// three-term recurrence (n P_n = (2n-1) x P_{n-1} - (n-1) P_{n-2}).
void gdg_gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        double wt = 2.0 / ((1.0 - z * z) * dp * dp);
        // map [-1,1] -> [0,1]; z > 0 for i < n/2 (descending)
        x[i] = 0.5 * (1.0 - z);
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[i] = w[n - 1 - i] = 0.5 * wt;
    }
}

static int stencil_first(int k, int p, int N) {
    int q = (p + 1) / 2;
    int s = k - q + 1;
    if (s < 0) s = 0;
    if (s > N - p) s = N - p;
    return s;
}

// phi_i(r), phi_i'(r) (d/dr on [0,1]) of all N+1 functions using the
// polynomial piece of `cell` (cell < 0: the cell containing r).  On cell k
// the basis is the Lagrange basis of the p+1 nodes s(k)..s(k)+p; nodes
// outside that stencil have zero functions there.
void gdg_eval_basis(int p, int N, double r, int cell, double *phi, double *dphi) {
    int k = cell;
    if (k < 0) {
        k = (int)std::floor(r * N);
        if (k < 0) k = 0;
        if (k > N - 1) k = N - 1;
    }
    for (int i = 0; i <= N; ++i) { phi[i] = 0.0; dphi[i] = 0.0; }
    int s = stencil_first(k, p, N);
    double h = 1.0 / N;
    for (int m = 0; m <= p; ++m) {
        double xm = (s + m) * h;
        double val = 1.0;
        for (int l = 0; l <= p; ++l) {
            if (l == m) continue;
            double xl = (s + l) * h;
            val *= (r - xl) / (xm - xl);
        }
        // derivative: sum over the dropped factor
        double der = 0.0;
        for (int kk = 0; kk <= p; ++kk) {
            if (kk == m) continue;
            double xk = (s + kk) * h;
            double term = 1.0 / (xm - xk);
            for (int l = 0; l <= p; ++l) {
                if (l == m || l == kk) continue;
                double xl = (s + l) * h;
                term *= (r - xl) / (xm - xl);
            }
            der += term;
        }
        phi[s + m] = val;
        dphi[s + m] = der;
    }
}

// Cholesky A = L L^T (lower, row-major n x n); returns false if not SPD.
static bool cholesky(int n, const double *A, double *L) {
    for (int i = 0; i < n * n; ++i) L[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
        if (!(d > 0.0)) return false;
        L[j * n + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = s / L[j * n + j];
        }
    }
    return true;
}

// Cyclic Jacobi eigen-solver for a symmetric matrix (in place: A becomes
// diagonal, V accumulates the rotations: A0 = V diag V^T).
static void jacobi_eigen(int n, double *A, double *V) {
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

int gdg_build_basis(int p, int N, std::vector<double> &M, std::vector<double> &S,
                    std::vector<double> &phiL, std::vector<double> &phiR,
                    std::vector<double> &dphiL, std::vector<double> &dphiR,
                    std::vector<double> &Psi, std::vector<double> &lam) {
    if (p < 1 || p % 2 == 0 || N < p) return GDG_EINVAL;
    int n1 = N + 1;
    if (n1 > GDG_MAXN1) return GDG_EUNSUPPORTED;
    M.assign(n1 * n1, 0.0);
    S.assign(n1 * n1, 0.0);
    std::vector<double> gx, gw, phi(n1), dphi(n1);
    gdg_gauss_legendre(p + 1, gx, gw);   // exact for the degree-2p integrands
    double h = 1.0 / N;
    for (int k = 0; k < N; ++k)
        for (int g = 0; g < p + 1; ++g) {
            double r = (k + gx[g]) * h, w = gw[g] * h;
            gdg_eval_basis(p, N, r, k, phi.data(), dphi.data());
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n1; ++b) {
                    M[a * n1 + b] += w * phi[a] * phi[b];
                    S[a * n1 + b] += w * dphi[a] * dphi[b];
                }
        }
    phiL.assign(n1, 0.0); phiR.assign(n1, 0.0); dphiL.assign(n1, 0.0); dphiR.assign(n1, 0.0);
    gdg_eval_basis(p, N, 0.0, 0, phiL.data(), dphiL.data());
    gdg_eval_basis(p, N, 1.0, N - 1, phiR.data(), dphiR.data());

    // generalized eigenproblem S psi = lambda M psi via M = L L^T
    std::vector<double> L(n1 * n1), Li(n1 * n1, 0.0), C(n1 * n1), Y(n1 * n1);
    if (!cholesky(n1, M.data(), L.data())) return GDG_EINVAL;
    for (int c = 0; c < n1; ++c) {          // Li = L^-1 by forward substitution
        for (int i = 0; i < n1; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * n1 + k] * Li[k * n1 + c];
            Li[i * n1 + c] = s / L[i * n1 + i];
        }
    }
    for (int i = 0; i < n1; ++i)            // C = Li S Li^T
        for (int j = 0; j < n1; ++j) {
            double s = 0.0;
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n1; ++b) s += Li[i * n1 + a] * S[a * n1 + b] * Li[j * n1 + b];
            C[i * n1 + j] = s;
        }
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < i; ++j) C[i * n1 + j] = C[j * n1 + i] = 0.5 * (C[i * n1 + j] + C[j * n1 + i]);
    jacobi_eigen(n1, C.data(), Y.data());
    std::vector<int> order(n1);
    for (int i = 0; i < n1; ++i) order[i] = i;
    for (int i = 0; i < n1; ++i)            // ascending eigenvalues (insertion sort)
        for (int j = i; j > 0 && C[order[j] * n1 + order[j]] < C[order[j - 1] * n1 + order[j - 1]]; --j)
            std::swap(order[j], order[j - 1]);
    Psi.assign(n1 * n1, 0.0);
    lam.assign(n1, 0.0);
    for (int k = 0; k < n1; ++k) {
        int c = order[k];
        lam[k] = C[c * n1 + c];
        for (int i = 0; i < n1; ++i) {      // psi = Li^T y
            double s = 0.0;
            for (int a = 0; a < n1; ++a) s += Li[a * n1 + i] * Y[a * n1 + c];
            Psi[i * n1 + k] = s;
        }
    }
    // exact constant mode (kernel of S), then M-orthonormalise the rest
    double oMo = 0.0;
    for (int a = 0; a < n1; ++a)
        for (int b = 0; b < n1; ++b) oMo += M[a * n1 + b];
    lam[0] = 0.0;
    for (int i = 0; i < n1; ++i) Psi[i * n1] = 1.0 / std::sqrt(oMo);
    auto mdot = [&](int k1, int k2) {
        double s = 0.0;
        for (int a = 0; a < n1; ++a)
            for (int b = 0; b < n1; ++b) s += Psi[a * n1 + k1] * M[a * n1 + b] * Psi[b * n1 + k2];
        return s;
    };
    for (int k = 1; k < n1; ++k) {
        for (int j = 0; j < k; ++j) {
            double c = mdot(j, k);
            for (int i = 0; i < n1; ++i) Psi[i * n1 + k] -= c * Psi[i * n1 + j];
        }
        double nrm = std::sqrt(mdot(k, k));
        // sign convention: largest-magnitude component positive
        int imax = 0;
        for (int i = 1; i < n1; ++i)
            if (std::fabs(Psi[i * n1 + k]) > std::fabs(Psi[imax * n1 + k]) + 1e-12) imax = i;
        double sg = Psi[imax * n1 + k] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < n1; ++i) Psi[i * n1 + k] *= sg / nrm;
    }
    return GDG_OK;
}

extern "C" int gdg_basis_1d(int p, int N, double *M, double *S, double *phiL, double *phiR,
                            double *dphiL, double *dphiR, double *Psi, double *lambda) {
    std::vector<double> vM, vS, a, b, c, d, vP, vl;
    int st = gdg_build_basis(p, N, vM, vS, a, b, c, d, vP, vl);
    if (st != GDG_OK) return st;
    int n1 = N + 1;
    auto cp = [](double *dst, const std::vector<double> &src) {
        if (dst) std::memcpy(dst, src.data(), src.size() * sizeof(double));
    };
    (void)n1;
    cp(M, vM); cp(S, vS); cp(phiL, a); cp(phiR, b); cp(dphiL, c); cp(dphiR, d);
    cp(Psi, vP); cp(lambda, vl);
    return GDG_OK;
}

// ------------------------------------------------------- profiling -------

cudaEvent_t Profiler::begin(cudaStream_t s) {
    while (pool.size() < used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
    }
    cudaEvent_t e0 = pool[used++];
    cudaEventRecord(e0, s);
    return e0;
}

void Profiler::end(int kind, cudaEvent_t start, cudaStream_t s) {
    cudaEvent_t e1 = pool[used++];
    cudaEventRecord(e1, s);
    recs.push_back({kind, {start, e1}});
}

void Profiler::clear() {
    recs.clear();
    used = 0;
}

void Profiler::destroy() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    clear();
}

extern "C" int gdg_profile_enable(gdg_ctx *ctx, int on) {
    if (!ctx) return GDG_EINVAL;
    cudaDeviceSynchronize();
    ctx->prof.clear();
    ctx->prof.on = on != 0;
    return GDG_OK;
}

extern "C" int gdg_profile_read(gdg_ctx *ctx, int kind, long long *launches, double *ms) {
    if (!ctx || !launches || !ms || kind < 0 || kind >= GDG_K_COUNT) return GDG_EINVAL;
    int st = gdg_cuda_check(ctx, cudaDeviceSynchronize(), "gdg_profile_read");
    if (st) return st;
    long long n = 0;
    double t = 0.0;
    for (auto &r : ctx->prof.recs) {
        if (r.first != kind) continue;
        float f = 0.f;
        if (cudaEventElapsedTime(&f, r.second.first, r.second.second) == cudaSuccess) {
            t += f;
            ++n;
        }
    }
    *launches = n;
    *ms = t;
    return GDG_OK;
}

// -------------------------------------------------------- context --------

static int validate(const gdg_problem *pb, std::string &why) {
    if (!pb) { why = "null problem"; return GDG_EINVAL; }
    if (pb->dim < 1 || pb->dim > 3) { why = "dim must be 1, 2 or 3"; return GDG_EINVAL; }
    if (pb->dim == 3 && pb->coef != GDG_COEF_CONST) { why = "3-D elements: GDG_COEF_CONST only"; return GDG_EUNSUPPORTED; }
    if (pb->dim == 3 && pb->N + 1 > 10) { why = "3-D elements: N+1 <= 10"; return GDG_EUNSUPPORTED; }
    if (pb->p < 1 || pb->p % 2 == 0) { why = "p must be odd and >= 1"; return GDG_EINVAL; }
    if (pb->N < pb->p) { why = "need N >= p"; return GDG_EINVAL; }
    if (pb->N + 1 > GDG_MAXN1) { why = "N+1 > 16 not supported"; return GDG_EUNSUPPORTED; }
    for (int k = 0; k < pb->dim; ++k) {
        if (pb->n_elem[k] < 1) { why = "n_elem must be >= 1"; return GDG_EINVAL; }
        if (!(pb->hi[k] > pb->lo[k])) { why = "need hi > lo"; return GDG_EINVAL; }
        if (pb->bc[k] != GDG_BC_DIRICHLET && pb->bc[k] != GDG_BC_PERIODIC) { why = "bad bc"; return GDG_EINVAL; }
    }
    if (pb->flux != GDG_FLUX_CENTRAL && pb->flux != GDG_FLUX_UPWIND && pb->flux != GDG_FLUX_ALTERNATING) {
        why = "bad flux";
        return GDG_EINVAL;
    }
    if (pb->coef == GDG_COEF_CONST) {
        if (!(pb->c2 > 0.0)) { why = "c2 must be > 0"; return GDG_EINVAL; }
        if (pb->solver != GDG_SOLVE_DIAG) { why = "constant coefficients use GDG_SOLVE_DIAG"; return GDG_EINVAL; }
        if (pb->route != GDG_ROUTE_MODAL && pb->route != GDG_ROUTE_NODAL) { why = "bad route"; return GDG_EINVAL; }
        if (pb->route == GDG_ROUTE_NODAL && pb->dim == 3) { why = "the nodal-state route: dim 1 and 2 only"; return GDG_EUNSUPPORTED; }
        if (pb->route == GDG_ROUTE_NODAL && (pb->rows[0] || pb->rows[1])) {
            why = "the nodal-state route: whole meshes only (no bands of rows)";
            return GDG_EUNSUPPORTED;
        }
        if (pb->precision != GDG_FP64) { why = "the diagonalised route has no solve to refine: FP64 only"; return GDG_EUNSUPPORTED; }
    } else if (pb->coef == GDG_COEF_NODAL) {
        if (pb->dim != 2) { why = "GDG_COEF_NODAL needs dim 2"; return GDG_EINVAL; }
        if (!pb->x_nodes || !pb->y_nodes || !pb->c2_nodes) { why = "null nodal arrays"; return GDG_EINVAL; }
        if (pb->solver != GDG_SOLVE_PCG && pb->solver != GDG_SOLVE_INVERSE) {
            why = "GDG_COEF_NODAL needs GDG_SOLVE_PCG or GDG_SOLVE_INVERSE";
            return GDG_EINVAL;
        }
        if (pb->solver == GDG_SOLVE_INVERSE && pb->precision != GDG_FP64) {
            why = "GDG_SOLVE_INVERSE has no iteration to refine: FP64 only";
            return GDG_EUNSUPPORTED;
        }
        if (pb->precond == GDG_PC_IC0) {
            why = "IC(0) preconditioning is not run on the GPU (sequential triangular solves per element); "
                  "use GDG_PC_FDM";
            return GDG_EUNSUPPORTED;
        }
        if (pb->precond != GDG_PC_FDM && pb->precond != GDG_PC_NONE) { why = "bad precond"; return GDG_EINVAL; }
        if (pb->pcg_maxit < 1 || !(pb->pcg_rtol >= 0.0)) { why = "bad PCG settings"; return GDG_EINVAL; }
        if (pb->nquad < 0 || pb->nquad > 12) { why = "nquad must be in 0..12"; return GDG_EINVAL; }
    } else {
        why = "bad coef";
        return GDG_EINVAL;
    }
    if (pb->precision == GDG_TF32 || pb->precision == GDG_BF16) {
        why = "TF32 / BF16 inner solves are not built: refinement needs kappa u_low < 1 and the u_t systems have "
              "kappa 1e3..1e5 (use GDG_MIXED, FP32 inner solves)";
        return GDG_EUNSUPPORTED;
    }
    if (pb->precision != GDG_FP64 && pb->precision != GDG_MIXED) { why = "bad precision"; return GDG_EINVAL; }
    if (pb->rows[0] || pb->rows[1]) {
        if (pb->dim != 2 || pb->coef != GDG_COEF_CONST) {
            why = "bands of rows (partitioned meshes): 2-D GDG_COEF_CONST only";
            return GDG_EUNSUPPORTED;
        }
        if (pb->rows[0] < 0 || pb->rows[1] <= pb->rows[0] || pb->rows[1] > pb->n_elem[1]) {
            why = "rows must satisfy 0 <= rows[0] < rows[1] <= n_elem[1]";
            return GDG_EINVAL;
        }
        const bool partial = pb->rows[0] > 0 || pb->rows[1] < pb->n_elem[1];
        if (partial && pb->bc[1] != GDG_BC_DIRICHLET) {
            why = "a band of rows needs bc[1] = GDG_BC_DIRICHLET (a periodic y direction is not split)";
            return GDG_EINVAL;
        }
    }
    return GDG_OK;
}

extern "C" int gdg_create(const gdg_problem *pb, gdg_ctx **out) {
    if (!out) return GDG_EINVAL;
    *out = nullptr;
    std::string why;
    int st = validate(pb, why);
    if (st != GDG_OK) {
        std::fprintf(stderr, "gdg_create: %s\n", why.c_str());
        return st;
    }
    gdg_ctx *ctx = new (std::nothrow) gdg_ctx();
    if (!ctx) return GDG_ENOMEM;
    ctx->pb = *pb;
    ctx->pb.x_nodes = ctx->pb.y_nodes = ctx->pb.c2_nodes = nullptr;
    ctx->dim = pb->dim;
    ctx->nx = pb->n_elem[0];
    ctx->ny = pb->dim >= 2 ? pb->n_elem[1] : 1;
    if (pb->dim == 2 && (pb->rows[0] || pb->rows[1])) ctx->ny = pb->rows[1] - pb->rows[0];   // a band of rows
    ctx->nz = pb->dim == 3 ? pb->n_elem[2] : 1;
    ctx->N = pb->N;
    ctx->n1 = pb->N + 1;
    ctx->p = pb->p;
    ctx->ne = ctx->nx * ctx->ny * ctx->nz;
    ctx->ndof = (long long)ctx->ne * (pb->dim == 3 ? ctx->n1 * ctx->n1 * ctx->n1
                                                   : (pb->dim == 2 ? ctx->n1 * ctx->n1 : ctx->n1));
    cudaGetDevice(&ctx->device);
    st = gdg_build_basis(ctx->p, ctx->N, ctx->Mh, ctx->Sh, ctx->phiL, ctx->phiR, ctx->dphiL,
                         ctx->dphiR, ctx->Psih, ctx->lamh);
    if (st == GDG_OK) {
        if (pb->coef == GDG_COEF_CONST) {
            st = gdg_const_setup(ctx);
        } else {
            ctx->pb.x_nodes = pb->x_nodes;   // read during setup only
            ctx->pb.y_nodes = pb->y_nodes;
            ctx->pb.c2_nodes = pb->c2_nodes;
            st = gdg_var_setup(ctx);
            ctx->pb.x_nodes = ctx->pb.y_nodes = ctx->pb.c2_nodes = nullptr;
        }
    }
    if (st != GDG_OK) {
        std::fprintf(stderr, "gdg_create: %s\n", ctx->err.c_str());
        gdg_destroy(ctx);
        return st;
    }
    *out = ctx;
    return GDG_OK;
}

extern "C" int gdg_destroy(gdg_ctx *ctx) {
    if (!ctx) return GDG_EINVAL;
    cudaDeviceSynchronize();
    gdg_const_free(ctx);
    gdg_var_free(ctx);
    ctx->prof.destroy();
    cudaFree(ctx->d_io);
    delete ctx;
    return GDG_OK;
}

extern "C" long long gdg_state_len(const gdg_ctx *ctx) { return ctx ? ctx->ndof : -1; }

static bool is_const(const gdg_ctx *ctx) { return ctx->pb.coef == GDG_COEF_CONST; }

extern "C" int gdg_rhs(gdg_ctx *ctx, const double *u, const double *v, double t, double *du, double *dv,
                       void *stream) {
    if (!ctx || !u || !v || !du || !dv || !std::isfinite(t)) return GDG_EINVAL;
    if (du == u || du == v || dv == u || dv == v)
        return gdg_set_err(ctx, GDG_EINVAL, "gdg_rhs: outputs alias inputs");
    cudaStream_t s = (cudaStream_t)stream;
    return is_const(ctx) ? gdg_const_rhs(ctx, u, v, du, dv, s) : gdg_var_rhs(ctx, u, v, t, du, dv, s);
}

extern "C" int gdg_mass_solve(gdg_ctx *ctx, int which, const double *b, double *x, void *stream) {
    if (!ctx || !b || !x) return GDG_EINVAL;
    if (which != GDG_OP_M && which != GDG_OP_S) return gdg_set_err(ctx, GDG_EINVAL, "bad operator");
    if (!is_const(ctx)) return gdg_set_err(ctx, GDG_EINVAL, "gdg_mass_solve needs GDG_COEF_CONST");
    return gdg_const_mass_solve(ctx, which, b, x, (cudaStream_t)stream);
}

extern "C" int gdg_pcg(gdg_ctx *ctx, int which, const double *b, double *x, gdg_pcg_stats *stats,
                       void *stream) {
    if (!ctx || !b || !x) return GDG_EINVAL;
    if (which != GDG_OP_M && which != GDG_OP_S) return gdg_set_err(ctx, GDG_EINVAL, "bad operator");
    if (is_const(ctx)) return gdg_set_err(ctx, GDG_EINVAL, "gdg_pcg needs GDG_COEF_NODAL");
    return gdg_var_pcg(ctx, which, b, x, stats, (cudaStream_t)stream);
}

extern "C" int gdg_step_stats(gdg_ctx *ctx, gdg_pcg_stats *u_sys, gdg_pcg_stats *v_sys) {
    if (!ctx) return GDG_EINVAL;
    if (is_const(ctx)) return gdg_set_err(ctx, GDG_EINVAL, "gdg_step_stats needs GDG_SOLVE_PCG");
    return gdg_var_step_stats(ctx, u_sys, v_sys);
}

extern "C" int gdg_step(gdg_ctx *ctx, double *u, double *v, double t0, double dt, int nsteps,
                        void *stream) {
    // t0 matters only with a point source (GDG_COEF_NODAL); otherwise the problem is autonomous
    if (!ctx || !u || !v || nsteps < 0 || !(dt > 0.0)) return GDG_EINVAL;
    if (nsteps == 0) return GDG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    return is_const(ctx) ? gdg_const_step(ctx, u, v, dt, nsteps, s)
                         : gdg_var_step(ctx, u, v, t0, dt, nsteps, s);
}

extern "C" int gdg_step_host(gdg_ctx *ctx, double *u, double *v, double t0, double dt, int nsteps,
                             void *stream) {
    if (!ctx || !u || !v || nsteps < 0 || !(dt > 0.0)) return GDG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)ctx->ndof * sizeof(double);
    int st;
    if (!ctx->d_io &&
        (st = gdg_cuda_check(ctx, cudaMalloc((void **)&ctx->d_io, 2 * bytes), "gdg_step_host alloc")))
        return st;
    double *du = ctx->d_io, *dv = ctx->d_io + ctx->ndof;
    st = gdg_cuda_check(ctx, cudaMemcpyAsync(du, u, bytes, cudaMemcpyHostToDevice, s), "h2d u");
    if (st == GDG_OK) st = gdg_cuda_check(ctx, cudaMemcpyAsync(dv, v, bytes, cudaMemcpyHostToDevice, s), "h2d v");
    if (st == GDG_OK) st = gdg_step(ctx, du, dv, t0, dt, nsteps, stream);
    if (st == GDG_OK) st = gdg_cuda_check(ctx, cudaMemcpyAsync(u, du, bytes, cudaMemcpyDeviceToHost, s), "d2h u");
    if (st == GDG_OK) st = gdg_cuda_check(ctx, cudaMemcpyAsync(v, dv, bytes, cudaMemcpyDeviceToHost, s), "d2h v");
    int st2 = gdg_cuda_check(ctx, cudaStreamSynchronize(s), "gdg_step_host sync");
    return st != GDG_OK ? st : st2;
}

extern "C" int gdg_energy(gdg_ctx *ctx, const double *u, const double *v, double *E, void *stream) {
    if (!ctx || !u || !v || !E) return GDG_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int st = is_const(ctx) ? gdg_const_energy(ctx, u, v, E, s) : gdg_var_energy(ctx, u, v, E, s);
    if (st == GDG_OK && !std::isfinite(*E)) return gdg_set_err(ctx, GDG_ENONFINITE, "energy is not finite");
    return st;
}

// ---------------------------------------------------- index checks ------

extern "C" int gdg_check_status(long long *count, int *site, long long *index, long long *bound, int reset) {
    if (count) *count = 0;
    if (site) *site = 0;
    if (index) *index = 0;
    if (bound) *bound = 0;
    if (!GDG_CHECKS) return GDG_EUNSUPPORTED;
    if (cudaDeviceSynchronize() != cudaSuccess) return GDG_ECUDA;
    int (*const readers[])(GdgCheckSlot *, int) = {gdg_checks_read_const, gdg_checks_read_const3, gdg_checks_read_var,
                                                   gdg_checks_read_batch};
    GdgCheckSlot acc{};
    for (auto rd : readers) {
        GdgCheckSlot s{};
        if (rd(&s, reset)) return GDG_ECUDA;
        if (s.count && !acc.count) acc = s;
        else acc.count += s.count;
    }
    if (count) *count = (long long)acc.count;
    if (site) *site = (int)acc.site;
    if (index) *index = acc.index;
    if (bound) *bound = acc.bound;
    return GDG_OK;
}
