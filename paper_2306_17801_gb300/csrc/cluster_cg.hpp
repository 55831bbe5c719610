// Whole-solve cluster kernels: argument block, per-system descriptors and
// launch helpers (see cluster_cg.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace apcg {

constexpr int kClusterThreads = 512;  // threads per CTA at most

// One SPD system of a (possibly single-system) batch.
struct SysDesc {
  int64_t row0;  // first row in the concatenated rowptr/b/x
  int32_t n;     // rows
  int32_t pad;
};

// Outcome of one system, written by the cluster that solved it.
struct SysResult {
  int32_t iters;  // CG iterations (refinement: inner iterations summed over corrections)
  int32_t done;   // kDone* of cg_internal.hpp
  double rr;      // (r,r) at the last convergence test (refinement: of the last float64 residual)
  double bnorm2;  // (b,b)
  int32_t outer;  // refinement: corrections applied (0 for CG)
  int32_t pad;
};

struct ClusterArgs {
  const int32_t* rowptr;  // global row pointers (nnz positions over the concatenation)
  const int32_t* col;     // column indices local to each system
  const double* val;      // float64 values, or nullptr (refinement: use val32 widened)
  const float* val32;     // float32 values (refinement), or nullptr (use val rounded)
  const double* dinv;     // precomputed 1/diag over the concatenation, or nullptr
  const double* b;
  double* x;
  const SysDesc* sys;
  const int32_t* order;   // solve order (longest first), or nullptr for 0..nsys-1
  int32_t nsys;
  int32_t check_every;
  unsigned int* next;     // work counter, zero at launch
  SysResult* res;
  double rtol, atol;
  int32_t max_it;         // CG: <= 0 means 10 n per system; refinement: inner iterations per correction
  int32_t hist_len;       // CG only: alpha/beta of iterations 1..hist_len of every system s, written to
  double* alpha_h;        // alpha_h[s * hist_len + i] and beta_h[s * hist_len + i] (nullptr when hist_len
  double* beta_h;         // is 0)
  // refinement only
  float rtol_inner;
  int32_t max_outer;
};

// Cluster size, threads per CTA, rows per thread and smem rows of a launch.
struct ClusterShape {
  int C = 1, tpb = kClusterThreads, R = 1, rpc_max = 1;
  bool ok = true;
  bool ir = false;  // mixed-precision refinement kernel (more shared memory per row)
};

int cluster_rows_per_cta(int n, int C);
ClusterShape cluster_shape_for(int n_max, int C, bool ir = false);
ClusterShape default_cluster_shape(int n, bool ir = false);
// The shape for C CTAs per cluster, halving C until the device can schedule it (ok = false if none).
ClusterShape schedulable_shape(int n_max, int C, bool ir = false);
// Launch the float64 CG kernel or, for sh.ir, the refinement kernel.
cudaError_t launch_cluster_cg(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s);
// Clusters of this shape that fit on the device at once (0: not schedulable).
int max_active_clusters(const ClusterShape& sh);

// Whole-solve Jacobi-TFQMR (cluster_tfqmr.cu): the launch shape for systems of
// up to n rows (ok = false above 16384 rows or if none is schedulable), and
// the launch (args as for CG; res receives iters, done, the squared bound as
// rr and ||D^-1 b||^2 as bnorm2).
ClusterShape tfqmr_cluster_shape(int n);
cudaError_t launch_cluster_tfqmr(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s);

}  // namespace apcg
