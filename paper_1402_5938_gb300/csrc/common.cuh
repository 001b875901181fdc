// Internal definitions shared by the translation units of libhmg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>

#include "../../include/hmg.h"

namespace hmg {

constexpr int kMaxN = 17;  // p <= 16

// Structured mesh of one level: nelem per axis, order p, nodes per axis (E p + 1).
struct Mesh {
  int dim;
  int E[3];
  int p;
  long long Nn[3];
  long long nelem;
  long long N;  // total nodes
};

// 1D tables of order p = N-1 (q = N Gauss points), in precision T.
//   B[q*N + a]  = l_a(g_q): GLL Lagrange basis a at Gauss point q (interpolation GLL -> Gauss)
//   D[q*N + s]  = l^G_s'(g_q): derivative of the Gauss-point Lagrange basis (collocated derivative)
template <int N, typename T>
struct Tab {
  T B[N * N];
  T D[N * N];
};

// Tables of the geometry and diagonal kernels (FP64 only).
//   Bd = D B (GLL basis derivative at Gauss points); r[a]: GLL nodes on [0,1];
//   w[q]: Gauss weights on [0,1];
//   BB/BD/DD[q*N+a] = B*B, B*Bd, Bd*Bd with Bd = D B (GLL basis derivative at Gauss points).
template <int N>
struct GeoTab {
  double B[N * N];
  double D[N * N];
  double Bd[N * N];
  double r[N];
  double w[N];
  double BB[N * N];
  double BD[N * N];
  double DD[N * N];
};

// Host-side 1D tables for one order (computed by host_basis.cu).
struct Basis1D {
  int p, n;
  double r[kMaxN], g[kMaxN], w[kMaxN];
  double B[kMaxN * kMaxN];   // [q][a]
  double D[kMaxN * kMaxN];   // [q][s]
  double Bd[kMaxN * kMaxN];  // [q][a]
};

void make_basis(int p, Basis1D* out);
// l_a(x) for the nodes r[0..n) (exactly 1/0 at a node); out[a], a < n
void lagrange_row(const double* r, int n, double x, double* out);
double hessenberg_max_real_eig(const double* H, int m);

void set_error(const std::string& msg);

// Streaming multiprocessors of the current device (queried once per device).
int device_sm_count();

// Number of kernels this library has launched (all threads); read by hmg_launch_count().
long long add_launches(long long n);
cudaError_t ensure_smem_ptr(const void* kernel, size_t bytes);
inline cudaError_t counted(cudaError_t e, long long n = 1) {
  if (e == cudaSuccess) add_launches(n);
  return e;
}

// Page-locked host blocks from a process-wide pool (pass the same size to pinned_free).
void* pinned_alloc(size_t bytes);
void pinned_free(void* p, size_t bytes);

// Device memory from the device's stream-ordered pool (no implicit device synchronization,
// unlike cudaMalloc / cudaFree); the first call on a device keeps freed memory cached in the pool.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

struct ProblemImpl;  // defined in problem.cuh
// Whether a problem can join a grouped batch plan (batch.cu).
bool batch_supported(const hmg_problem* p);

}  // namespace hmg

#define HMG_CUDA_TRY(expr)                                                          \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      ::hmg::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));         \
      return HMG_EDEVICE;                                                           \
    }                                                                               \
  } while (0)
