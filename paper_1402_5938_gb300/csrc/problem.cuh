// Internal state of a problem handle: the multigrid hierarchy (per-level meshes, tables,
// geometric factors, smoother data, transfer stencils, coarsest inverse) and the solve buffers and
// graphs, shared by the translation units that drive solves (hmg.cu, batch.cu).
#pragma once

#include <vector>

#include "common.cuh"
#include "ops.cuh"
#include "vector.cuh"

namespace hmg {

struct Level {
  Mesh m{};
  Basis1D basis{};
  long long nI = 0;       // interior nodes
  double* G = nullptr;    // [E][NC][NP] geometric factors mu w detJ J^-1 J^-T
  double* wdetJ = nullptr;
  double* dinv = nullptr;
  void* Glow = nullptr;   // factors of the mixed V-cycle's operator (FP32, FP16 or BF16, grouped layout)
  double* Ke = nullptr;   // element matrices of a low-order FP64 level (dense-apply variant)
  double* Kb = nullptr;   // block Jacobi: inverses of the element-interior blocks [E][MI][MI]
  double* dinv_s = nullptr;  // block Jacobi: D^-1 on shared nodes, 0 at element-interior nodes
  float* gsc = nullptr;   // 16-bit factors: per-element power-of-two scales
  Tc16Data tc{};          // tensor-core form of the 16-bit apply: its factor layout, Phi image, v scale
  void* Gdf = nullptr;    // finest level, double-float operator: G split into float pairs
  float* dinv32 = nullptr;
  double lam = 0.0;       // Chebyshev bound
  int v64 = 0, v32 = 0;   // apply variants chosen by the autotuner (v32: of the V-cycle
                          // operator, FP32 or 16-bit)
  double *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *d32 = nullptr;
  Axis1D P[3]{}, PT[3]{};  // transfer to the next coarser level: P rows fine, PT rows coarse
  double* Ainv = nullptr;  // coarsest: dense inverse of the interior operator
  long long* gmap = nullptr;
};

struct ProblemImpl {
  hmg_desc desc{};
  int device = 0;
  std::vector<Level> L;
  double* S = nullptr;        // device scalars
  double* X0 = nullptr;       // user node coordinates of the finest level [dim][N0] (node_xyz), else null
  int* err = nullptr;         // device error flag written by bounded waits in kernels
  double* partial = nullptr;  // reduction partials
  double* hostS = nullptr;    // pinned host copy of a scalar
  void* t1 = nullptr;         // transfer intermediates
  void* t2 = nullptr;
  double *pr = nullptr, *pz = nullptr, *pp = nullptr, *ph = nullptr;
  double *hx = nullptr, *hy = nullptr;  // finest-level staging of the host-buffer entry points
  std::vector<void*> dev_allocs;
  size_t bytes = 0;
  long long fine_applies = 0;
  // graph solves: one instantiated graph per mode (MG, PCG) with a device-side WHILE loop
  double* gb = nullptr;       // masked right-hand side
  double* gu = nullptr;       // solution
  int* ctrl = nullptr;        // iteration, status, maxit, history capacity
  double* hist = nullptr;     // residual history (capacity hist_cap + 1)
  int hist_cap = 0;
  int* host_ctrl = nullptr;   // pinned
  double* host_hist = nullptr;  // pinned
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  long long gkern[2][3] = {};  // kernel nodes per graph section: prologue, loop body (part 1), PCG part 2
  // lockstep graphs of batched solves (no conditional nodes, so different problems overlap):
  // [mode][0] prologue, [mode][1] first iteration half (PCG), [mode][2] one iteration
  cudaGraphExec_t lexec[2][3] = {};
  long long lkern[2][3] = {};
  bool capturing = false;

  // Device allocation from the stream-ordered pool, zeroed in order on the setup stream (the
  // caller's stream may be a non-blocking stream that the legacy default stream does not order
  // against); no implicit device synchronization, so setups overlap other streams' work.
  cudaStream_t setup_stream = nullptr;
  cudaStream_t own = nullptr;  // private stream on which destruction returns the memory
  cudaError_t alloc(void** p, size_t nbytes) {
    *p = nullptr;
    if (nbytes == 0) nbytes = 16;
    cudaError_t e = dev_alloc(p, nbytes, setup_stream);
    if (e != cudaSuccess) return e;
    dev_allocs.push_back(*p);
    bytes += nbytes;
    return cudaMemsetAsync(*p, 0, nbytes, setup_stream);
  }
  ~ProblemImpl() {
    for (int m = 0; m < 2; ++m) {
      if (gexec[m]) cudaGraphExecDestroy(gexec[m]);
      if (graph[m]) cudaGraphDestroy(graph[m]);
      for (int k = 0; k < 3; ++k)
        if (lexec[m][k]) cudaGraphExecDestroy(lexec[m][k]);
    }
    // callers finish their work on the problem first; work on the legacy default stream is
    // waited for here, then the memory goes back to the pool without a device-wide barrier
    cudaStreamSynchronize(nullptr);
    if (cap_stream) {
      cudaStreamSynchronize(cap_stream);
      cudaStreamDestroy(cap_stream);
    }
    cudaStream_t fs = own;
    for (void* p : dev_allocs) dev_free(p, fs);
    dev_free(hist, fs);
    if (fs) {
      cudaStreamSynchronize(fs);
      cudaStreamDestroy(fs);
    } else {
      cudaStreamSynchronize(nullptr);
    }
    pinned_free(hostS, 16 * sizeof(double));
    pinned_free(host_ctrl, 4 * sizeof(int));
    pinned_free(host_hist, (size_t)(hist_cap + 1) * sizeof(double));
  }
};

}  // namespace hmg

struct hmg_problem {
  hmg::ProblemImpl impl;
};
