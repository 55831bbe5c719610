// The Krylov core shared by the float64 CG solver and the float32 inner solver
// of mixed-precision refinement: device resources of one Jacobi-PCG solve,
// launch shapes, and launchers for the three iteration kernels and for the
// captured k-iteration graph (cg_core.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "apcg_internal.hpp"
#include "cg_internal.hpp"
#include "sell.cuh"
#include "stencil.cuh"

namespace apcg {

template <class T>
struct CgCore {
  int32_t n = 0;          // rows
  int32_t k = 1;          // convergence test every k iterations
  int32_t max_it = 0;
  int32_t hist_len = 0;
  int grid_spmv = 1, grid_vec = 1;
  dev::SellView<T> A;     // sliced-ELL copy of the matrix (values in T)
  dev::StencilView S;     // or the stencil operator (matrix-free plans: S.n == n > 0)
  T* dinv = nullptr;
  T* r = nullptr;
  T* p = nullptr;
  T* w = nullptr;
  T* z = nullptr;
  T* partials = nullptr;  // [3 * kMaxPartials]
  double* alpha_h = nullptr;
  double* beta_h = nullptr;
  CgState* st = nullptr;  // device state block (scalars stored as double)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  T* graph_x = nullptr;
  int32_t body = 1;  // iterations captured in one body of the conditional while node
  bool pdl = false;  // launch K1-K3 as programmatic dependents of their predecessor (launches one by one)
};

// Choose the persistent grids for n rows (nnz is informational).  Call after c.A is set.
template <class T>
void core_configure(CgCore<T>& c, int64_t nnz, int sms);

// K1: w = A p, gamma = (p,w); the last block forms alpha (device mode) or only gamma (host mode).
template <class T>
apcg_status core_k1(const CgCore<T>& c, T* x, cudaStream_t s, bool host);
// K2: x += alpha p, r -= alpha w, z = D^-1 r, (r,z), (r,r) on test iterations; test and beta.
template <class T>
apcg_status core_k2(const CgCore<T>& c, T* x, cudaStream_t s, bool host, double alpha,
                    cudaGraphConditionalHandle cond, int use_cond);
// K3: p = z + beta p.
template <class T>
apcg_status core_k3(const CgCore<T>& c, T* x, cudaStream_t s, bool host, double beta);
// Capture k iterations into the body of a conditional while node (once per x pointer).
template <class T>
apcg_status core_build_graph(CgCore<T>& c, T* x, cudaStream_t upload);
template <class T>
void core_release_graph(CgCore<T>& c);

// Set-up of the float64 solve: r = b - A x, z = D^-1 r, p = z, state initialised.
apcg_status core_setup_f64(const CgCore<double>& c, const double* b, double* x, double rtol, double atol,
                           cudaStream_t s);

}  // namespace apcg
