// Device-resident state of the Krylov solvers.
#pragma once

#include "common.cuh"

constexpr int KRYLOV_MAX_M = 64;   // largest GMRES cycle dimension (restart length + augmentation vectors)

struct KrylovState {
    // parameters
    double tol;
    int maxiter;
    int m;
    double2* partials;              // reduction scratch (nb x 32 complex)
    unsigned counter;               // last-block ticket of the running reduction
    // control
    int halt;                       // queued kernels return immediately when set
    int done;                       // the solve has finished (status is final)
    int status;                     // ss_status
    int iters;
    int sconv;                      // BiCGSTAB: converged on the half step s
    int k;                          // GMRES: inner steps in the current cycle
    // scalars
    double rnorm, snorm, rhat_norm, hnorm;
    double dnorm;                   // LGMRES: ||Z y|| of the last cycle's correction
    double2 rho, alpha, omega, beta;
    // GMRES
    double2 H[(KRYLOV_MAX_M + 1) * KRYLOV_MAX_M];   // row-major (i, j) at i * M + j
    double2 g[KRYLOV_MAX_M + 1];
    double2 y[KRYLOV_MAX_M];
    double2 hwork[KRYLOV_MAX_M + 1];
    double cs[KRYLOV_MAX_M];
    double2 sn[KRYLOV_MAX_M];
};

struct KrylovWork {
    int64_t n = 0;
    int method = 0;
    int m = 0;
    int kaug = 0;
    KrylovState* st = nullptr;
    KrylovState* host_st = nullptr;     // pinned mirror
    double2* partials = nullptr;
    double2* vecs = nullptr;
    size_t nvec = 0;
};

struct KrylovResultHost {
    int status = 0;
    int iters = 0;
    double resid = 0.0;
};

// Inverse-power inner solves may stop as soon as their iterate, normalised
// to unit trace, already satisfies ||L rho||_2 <= tol (checked by the host
// after each batch of queued iterations).
struct OuterCheck {
    const DeviceCSR* A = nullptr;     // L - sigma I (permuted)
    double sigma = 0.0;
    int64_t d = 0;
    const int32_t* tidx = nullptr;    // permuted positions of the diagonal elements
    double2* y = nullptr;             // scratch vector (n)
    double* scratch = nullptr;
    double2* trace = nullptr;         // device scalar
    double tol = 0.0;
};

// GMRES workspace: m + kaug + 1 basis vectors, m + kaug search directions
// (the last kaug hold LGMRES's stored corrections) and, with kaug > 0, one
// correction vector.
ss_status krylov_workspace(ss_ctx ctx, KrylovWork& w, int64_t n, int method, int m, int kaug = 0);
void krylov_workspace_free(ss_ctx ctx, KrylovWork& w);
ss_status bicgstab_dev(ss_ctx ctx, const DeviceCSR& A, ss_prec M, KrylovWork& w, const double2* b, double2* x,
                       double tol, int maxiter, KrylovResultHost* out, const OuterCheck* oc = nullptr);
// FP32 BiCGSTAB (inner solve of the mixed path): A's FP32 values, M's FP32 factors.
ss_status bicgstab_dev32(ss_ctx ctx, const DeviceCSR& A, const float2* val32, ss_prec M, KrylovWork& w,
                         const float2* b, float2* x, double tol, int maxiter, KrylovResultHost* out);
// Restarted GMRES(m), or LGMRES(m, kaug) for kaug > 0 (the workspace must
// have been made with the same m and kaug).
ss_status gmres_dev(ss_ctx ctx, const DeviceCSR& A, ss_prec M, KrylovWork& w, const double2* b, double2* x, double tol,
                    int maxiter, int m, KrylovResultHost* out, const OuterCheck* oc = nullptr, int kaug = 0);
