// Driver-side vector helpers (solver_util.cu).
#pragma once

#include "common.cuh"

ss_status su_zero(ss_ctx ctx, int64_t n, double2* v);
ss_status su_start_vector(ss_ctx ctx, int64_t n, uint64_t seed, const int32_t* perm_dev, double2* x);
ss_status su_normalise(ss_ctx ctx, int64_t n, double2* x, double* scratch);
ss_status su_trace(ss_ctx ctx, int64_t d, const int32_t* tidx, const double2* x, double2* out);
ss_status su_lrho(ss_ctx ctx, const DeviceCSR& A, const double2* x, int mode, double w_or_sigma, int64_t r0,
                  int64_t d, const int32_t* tidx, double2* y, double* scratch, double2* trace_dev, double* out,
                  double2* trace_host);
// Warm start: x[r] = rho[perm[r]] / tr(rho) (rho: natural column-major order,
// device), or x = 0 when tr(rho) = 0; trace_dev is scratch (one value).
ss_status su_warm_start(ss_ctx ctx, int64_t n, int64_t d, const int32_t* perm_dev, const double2* rho_dev,
                        double2* trace_dev, double2* x);
ss_status su_finalise(ss_ctx ctx, int64_t n, const int32_t* perm_dev, const double2* x, const double2* trace_dev,
                      double2* rho_dev);
ss_status su_condest(ss_ctx ctx, ss_prec M, int64_t n, double2* ones, double2* z, double* scratch, double* out);
int su_scratch_doubles();
// Mixed-precision refinement: r = b - A x in FP64, b32 = r / ||r||, x32 = 0;
// then x += ||r|| c.
ss_status su_refine_residual(ss_ctx ctx, const DeviceCSR& A, const double2* b, const double2* x, double2* y,
                             double2* r, float2* b32, float2* x32, double* scratch, double* rnorm);
ss_status su_refine_update(ss_ctx ctx, int64_t n, double2* x, const double* scratch, const float2* c);
