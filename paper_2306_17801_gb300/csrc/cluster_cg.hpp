// Whole-solve cluster kernel: argument block, per-system descriptors and
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
  int32_t iters;
  int32_t done;   // kDone* of cg_internal.hpp
  double rr;      // (r,r) at the last convergence test
  double bnorm2;  // (b,b)
};

struct ClusterArgs {
  const int32_t* rowptr;  // global row pointers (nnz positions over the concatenation)
  const int32_t* col;     // column indices local to each system
  const double* val;
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
  int32_t max_it;         // <= 0: 10 n per system
  int32_t hist_len;       // alpha/beta history of the first system in order
  double* alpha_h;
  double* beta_h;
};

// Cluster size, threads per CTA, rows per thread and smem rows of a launch.
struct ClusterShape {
  int C = 1, tpb = kClusterThreads, R = 1, rpc_max = 1;
  bool ok = true;
};

int cluster_rows_per_cta(int n, int C);
ClusterShape cluster_shape_for(int n_max, int C);
ClusterShape default_cluster_shape(int n);
// The shape for C CTAs per cluster, halving C until the device can schedule it (ok = false if none).
ClusterShape schedulable_shape(int n_max, int C);
cudaError_t launch_cluster_cg(const ClusterArgs& args, const ClusterShape& sh, int nclusters, cudaStream_t s);
// Clusters of this shape that fit on the device at once (0: not schedulable).
int max_active_clusters(const ClusterShape& sh);

}  // namespace apcg
