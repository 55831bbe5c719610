// Solver state and plan layout shared by the CG translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "apcg_internal.hpp"
#include "cluster_cg.hpp"

namespace apcg {

// 'done' word of the device state block.
enum : int32_t { kDoneRunning = 0, kDoneConverged = 1, kDoneNotConverged = 2, kDoneBreakdown = 3, kDoneBadDiagonal = 4 };

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

// The library context used by entry points that take host buffers.
apcg_ctx host_api_ctx();

// Forget a registration (mutex held by the caller).
void reg_forget_memory(const void* p);

apcg_status cg_plan_create(apcg_ctx ctx, apcg_mat A, const apcg_cg_opts* opts, apcg_cg_plan* out);
apcg_status cg_plan_destroy(apcg_cg_plan P);
apcg_status cg_plan_enqueue(apcg_cg_plan P, apcg_vec b, apcg_vec x);
apcg_status cg_plan_finish(apcg_cg_plan P, apcg_cg_result* res);

}  // namespace apcg

struct apcg_cg_plan_s {
  apcg_ctx ctx = nullptr;
  apcg_mat_s A;          // copy of the (non-owning) matrix view
  apcg_cg_opts opts;
  int32_t n = 0, k = 1, max_it = 0, hist_len = 0, mode = APCG_MODE_ASYNC_GRAPH, u = 8;
  int grid_spmv = 1, grid_vec = 1;
  char* ws = nullptr;    // workspace block (stream-ordered allocation)
  double *dinv = nullptr, *r = nullptr, *p = nullptr, *w = nullptr, *z = nullptr, *partials = nullptr;
  double *alpha_h = nullptr, *beta_h = nullptr;
  apcg::CgState* st = nullptr;       // device
  apcg::CgState* st_host = nullptr;  // pinned mirror
  apcg_id id = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double* graph_x = nullptr;
  bool pending = false;
  int64_t last_launches = 0;
  // whole-solve cluster mode
  apcg::ClusterShape shape;
  apcg::SysDesc* sys = nullptr;          // device, one entry
  unsigned int* next = nullptr;          // device work counter
  apcg::SysResult* sres = nullptr;       // device
  apcg::SysResult* sres_host = nullptr;  // pinned
};
