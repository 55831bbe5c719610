// Solver state and plan layout shared by the CG translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "apcg_internal.hpp"
#include "cluster_cg.hpp"
#include "stencil.cuh"

namespace apcg {

// 'done' word of the device state block.
enum : int32_t {
  kDoneRunning = 0,
  kDoneConverged = 1,
  kDoneNotConverged = 2,
  kDoneBreakdown = 3,
  kDoneBadDiagonal = 4,
  kDoneTimeout = 5  // a bounded device wait ran out (the staged float32 SpMV)
};

// Device-resident scalars of one solve (the managed scalars of Sec. 3.2).
struct CgState {
  double rho;      // (r,z) of the current residual
  double rho_new;  // (r,z) after the update (host-synchronous form)
  double alpha, beta, gamma;
  double rr;       // (r,r)
  double bnorm2;   // (b,b)
  double tol;      // max(rtol * ||b||, atol)
  int32_t iter;    // completed iterations
  int32_t done;    // kDone*
  int32_t max_it, check_every, hist_len;
  int32_t body_runs;   // executions of the graph body
  unsigned int ticket; // grid-reduction arrival counter
  int32_t pad;
};

// Launch the A0 kernel dinv = 1 / diag(A) (flags bad diagonals on ctx).
apcg_status launch_jacobi_setup(apcg_ctx ctx, apcg_mat A, double* dinv);
// y[0..n) = v on ctx's stream.
apcg_status launch_fill(apcg_ctx ctx, double* y, int64_t n, double v);

// The device description of a stencil operator (stencil.cu) and its centre weight (0 if it has no centre term).
const dev::StencilView& stencil_view(const apcg_stencil_s* S);
double stencil_center(const apcg_stencil_s* S);

// The library context used by entry points that take host buffers.
apcg_ctx host_api_ctx();

// Forget a registration (mutex held by the caller).
void reg_forget_memory(const void* p);


}  // namespace apcg
