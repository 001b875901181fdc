// Grouped batched solves: many independent problems (different meshes, coefficients, right-hand
// sides) solved by one CUDA graph whose every launch serves all problems of a group at once.
//
// Problems whose hierarchies have the same structure -- dimension, number of levels, order per
// level, smoother, nu_pre / nu_post, V-cycle precision -- form a group. Per level, a group keeps
// its members' vectors in one "super-vector" (each member's segment padded to 256 entries), so
// every elementwise smoother / PCG step is one launch over the whole group whose blocks look up
// their member and that member's scalars (Chebyshev coefficients from its own lambda_max, PCG
// alpha and beta, its active flag). Operator applies, transfers and the coarsest solve take
// per-member descriptors (mesh, factors, stencils, inverse) through a block -> (member, work
// unit) table, so one launch runs every member's elements. Dot products are segmented: one
// partial per 256-entry chunk, then a fixed-order sum per member.
//
// The solve is Algorithm 1 (or the MG iteration of Sec. 4.3) per member, in lockstep: one graph
// launch runs the prologue, then a device-side WHILE loop whose body applies the operator,
// updates and tests every active member; a member that converges (or reaches maxit, or goes
// non-finite) is switched inactive and its blocks return at once from then on, so its result is
// the one it would reach alone. Groups run as parallel branches of the graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "dispatch.cuh"
#include "element.cuh"
#include "ops.cuh"
#include "pencil.cuh"
#include "problem.cuh"
#include "vector.cuh"

namespace hmg {

namespace {

constexpr int kChunk = 256;  // entries per chunk of a segment; threads of the vector kernels

// one member's level (device side)
struct BLev {
  Mesh m;
  long long off;          // the member's segment in the level's super-vectors
  const double* G;        // FP64 factors [E][NC][NP]
  const void* Glow;       // reduced-precision factors (grouped layout)
  const void* Gdf;        // finest level, double-float operator: the FP64 factors as float pairs
  const float* gsc;
  const double* Ainv;     // coarsest level: dense inverse of the interior operator
  const long long* gmap;  // interior -> global node
  long long nI;
};

// one member's 1D transfer pass along `axis` (device side)
struct BPass {
  long long in_off, out_off;
  long long od[3];
  int axis, n_in;
  const int* rowptr;
  const int* col;
  const double* val;
  const float* val32;
};

__device__ __forceinline__ double warp_sum_b(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double block_sum_b(double v) {  // blockDim.x == kChunk; valid in thread 0
  __shared__ double red[kChunk / 32];
  v = warp_sum_b(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < kChunk / 32 ? red[lane] : 0.0;
    s = warp_sum_b(s);
  }
  return s;
}

// ---- operator applies: one block per (member, work unit) entry ----
template <int DIM, int N, int V>
__global__ void __launch_bounds__(Apply64Cfg<DIM, N, V>::GT)
kb_apply64(const double* __restrict__ X, double* __restrict__ Y, const BLev* __restrict__ lev,
           const int2* __restrict__ tab, const int* __restrict__ gid, const int* __restrict__ active,
           const __grid_constant__ Tab<N, double> t1d, const double alpha, const int amode, int* __restrict__ err) {
  const int2 w = tab[blockIdx.x];
  if (!active[gid[w.x]]) return;
  const BLev& L = lev[w.x];
  extern __shared__ __align__(128) unsigned char smem_b64[];
  apply64_tile<DIM, N, V>(X + L.off, Y + L.off, L.G, L.m, t1d, alpha, amode, err, (long long)w.y, smem_b64);
}

template <int DIM, int N, typename GT>
__global__ void __launch_bounds__(PencilCfg<DIM, N>::THREADS)
kb_apply_low(const float* __restrict__ X, float* __restrict__ Y, const BLev* __restrict__ lev,
             const int2* __restrict__ tab, const int* __restrict__ gid, const int* __restrict__ active,
             const __grid_constant__ PencilTab<N, float> t1d, const float alpha) {
  const int2 w = tab[blockIdx.x];
  if (!active[gid[w.x]]) return;
  const BLev& L = lev[w.x];
  extern __shared__ __align__(16) float smem_blow[];
  pencil_tile<DIM, N, GT, 2>(X + L.off, Y + L.off, static_cast<const GT*>(L.Glow), L.gsc, L.m, t1d, alpha,
                             (long long)w.y, smem_blow);
}

// the finest FP64 operator in double-float arithmetic (members built with fp64_arith = df64)
template <int DIM, int N>
__global__ void __launch_bounds__(PencilCfg<DIM, N, df64>::THREADS)
kb_apply_df64(const double* __restrict__ X, double* __restrict__ Y, const BLev* __restrict__ lev,
              const int2* __restrict__ tab, const int* __restrict__ gid, const int* __restrict__ active,
              const __grid_constant__ PencilTab<N, df64> t1d, const df64 alpha) {
  const int2 w = tab[blockIdx.x];
  if (!active[gid[w.x]]) return;
  const BLev& L = lev[w.x];
  extern __shared__ __align__(16) unsigned char smem_bdf[];
  pencil_tile<DIM, N, df64, 2, df64, double>(X + L.off, Y + L.off, static_cast<const df64*>(L.Gdf), nullptr, L.m,
                                             t1d, alpha, (long long)w.y, reinterpret_cast<df64*>(smem_bdf));
}

// ---- elementwise steps over super-vectors: one block per chunk, chunk -> member ----
#define KB_PROLOGUE                                  \
  const int mem = cmem[blockIdx.x];                  \
  if (!active[gid[mem]]) return;                     \
  const long long i = (long long)blockIdx.x * kChunk + threadIdx.x;

template <typename T>
__global__ void __launch_bounds__(kChunk)
kb_cheb_first(T* __restrict__ x, T* __restrict__ d, const T* __restrict__ b, const T* __restrict__ dinv,
              T* __restrict__ r, const double* __restrict__ inv_theta, const int* __restrict__ cmem,
              const int* __restrict__ gid, const int* __restrict__ active) {
  KB_PROLOGUE
  const T bi = b[i];
  const T v = dinv[i] * bi * (T)inv_theta[mem];
  d[i] = v;
  x[i] = v;
  if (r) r[i] = bi;
}
template <typename T>
__global__ void __launch_bounds__(kChunk)
kb_cheb(T* __restrict__ x, T* __restrict__ d, T* __restrict__ r, const T* __restrict__ b, const T* __restrict__ dinv,
        const double* __restrict__ c1, const double* __restrict__ c2, const int reset, const int* __restrict__ cmem,
        const int* __restrict__ gid, const int* __restrict__ active) {
  KB_PROLOGUE
  const T v = fma((T)c1[mem], d[i], (T)c2[mem] * dinv[i] * r[i]);
  d[i] = v;
  x[i] += v;
  if (reset) r[i] = b[i];
}
template <typename T>
__global__ void __launch_bounds__(kChunk)
kb_jacobi_first(T* __restrict__ x, const T* __restrict__ b, const T* __restrict__ dinv, T* __restrict__ r,
                const double* __restrict__ omega, const int* __restrict__ cmem, const int* __restrict__ gid,
                const int* __restrict__ active) {
  KB_PROLOGUE
  const T bi = b[i];
  x[i] = (T)omega[mem] * dinv[i] * bi;
  if (r) r[i] = bi;
}
template <typename T>
__global__ void __launch_bounds__(kChunk)
kb_jacobi(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ b, const T* __restrict__ dinv,
          const double* __restrict__ omega, const int reset, const int* __restrict__ cmem, const int* __restrict__ gid,
          const int* __restrict__ active) {
  KB_PROLOGUE
  x[i] = fma((T)omega[mem] * dinv[i], r[i], x[i]);
  if (reset) r[i] = b[i];
}
__global__ void __launch_bounds__(kChunk)
kb_axpy(double* __restrict__ u, const double* __restrict__ z, const int* __restrict__ cmem,
        const int* __restrict__ gid, const int* __restrict__ active) {
  KB_PROLOGUE
  u[i] += z[i];
}
// partial[chunk] = sum over the chunk of x y (0 for inactive members)
template <typename TX>
__global__ void __launch_bounds__(kChunk)
kb_dot(const TX* __restrict__ x, const TX* __restrict__ y, double* __restrict__ partial, const int* __restrict__ cmem,
       const int* __restrict__ gid, const int* __restrict__ active) {
  const int mem = cmem[blockIdx.x];
  const long long i = (long long)blockIdx.x * kChunk + threadIdx.x;
  double v = 0.0;
  if (active[gid[mem]]) v = (double)x[i] * (double)y[i];
  v = block_sum_b(v);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}
// PCG update with the member's alpha = rho / (p, A p); partial <- ||r||^2 per chunk
__global__ void __launch_bounds__(kChunk)
kb_pcg_update(double* __restrict__ u, double* __restrict__ r, const double* __restrict__ p,
              const double* __restrict__ h, const double* __restrict__ rho, const double* __restrict__ ph,
              double* __restrict__ partial, const int* __restrict__ cmem, const int* __restrict__ gid,
              const int* __restrict__ active) {
  const int mem = cmem[blockIdx.x];
  const int g = gid[mem];
  const long long i = (long long)blockIdx.x * kChunk + threadIdx.x;
  double acc = 0.0;
  if (active[g]) {
    const double alpha = ph[g] != 0.0 ? rho[g] / ph[g] : 0.0;  // p = 0 (zero right-hand side): no step
    u[i] = fma(alpha, p[i], u[i]);
    const double ri = fma(-alpha, h[i], r[i]);
    r[i] = ri;
    acc = ri * ri;
  }
  acc = block_sum_b(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}
__global__ void __launch_bounds__(kChunk)
kb_pcg_dir(double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ beta,
           const int* __restrict__ cmem, const int* __restrict__ gid, const int* __restrict__ active) {
  KB_PROLOGUE
  p[i] = fma(beta[gid[mem]], p[i], z[i]);
}
#undef KB_PROLOGUE

// Per-member sums of the chunk partials (fixed order) and what the iteration does with them.
enum SegOp : int { SEG_STORE = 0, SEG_RHO_BETA = 1, SEG_NEG_RATIO = 2 };
__global__ void kb_seg_finish(const double* __restrict__ partial, const int* __restrict__ cstart, int nmem,
                              const int* __restrict__ gid, const int* __restrict__ active, int op,
                              double* __restrict__ out, double* __restrict__ aux) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmem) return;
  const int g = gid[m];
  if (!active[g]) return;
  double acc = 0.0;
  for (int c = cstart[m]; c < cstart[m + 1]; ++c) acc += partial[c];
  if (op == SEG_STORE) out[g] = acc;
  else if (op == SEG_RHO_BETA) {  // out = rho (old -> new), aux = beta
    aux[g] = acc / out[g];
    out[g] = acc;
  } else {                        // out = beta = -acc / aux (aux = (p, A p))
    out[g] = aux[g] != 0.0 ? -acc / aux[g] : 0.0;
  }
}

// ---- transfers and the coarsest solve ----
template <typename T, typename V>
__global__ void __launch_bounds__(kChunk)
kb_axis(const T* __restrict__ in_base, T* __restrict__ out_base, const BPass* __restrict__ pass,
        const int2* __restrict__ tab, int mask_in, int mask_out, int acc, const int* __restrict__ gid,
        const int* __restrict__ active) {
  const int2 w = tab[blockIdx.x];
  if (!active[gid[w.x]]) return;
  const BPass& P = pass[w.x];
  const unsigned o0 = (unsigned)P.od[0], o1 = (unsigned)P.od[1], o2 = (unsigned)P.od[2];
  const unsigned t = (unsigned)w.y + threadIdx.x;
  if (t >= o0 * o1 * o2) return;
  const V* val = std::is_same<V, float>::value ? reinterpret_cast<const V*>(P.val32) : reinterpret_cast<const V*>(P.val);
  axis_point<T, V>(in_base + P.in_off, out_base + P.out_off, t, o0, o1, o2, P.axis, P.n_in, P.rowptr, P.col, val,
                   mask_in, mask_out, acc);
}

// x[gmap[i]] = sum_j Ainv[i][j] b[gmap[j]], one warp per row, 8 rows per block
template <typename T>
__global__ void __launch_bounds__(256)
kb_coarse(const T* __restrict__ B, T* __restrict__ X, const BLev* __restrict__ lev, const int2* __restrict__ tab,
          const int* __restrict__ gid, const int* __restrict__ active) {
  const int2 w = tab[blockIdx.x];
  if (!active[gid[w.x]]) return;
  const BLev& L = lev[w.x];
  const long long i = (long long)w.y + (threadIdx.x >> 5);
  if (i >= L.nI) return;
  const int lane = threadIdx.x & 31;
  const T* b = B + L.off;
  const double* row = L.Ainv + i * L.nI;
  double acc = 0.0;
  for (long long j = lane; j < L.nI; j += 32) acc = fma(row[j], (double)b[L.gmap[j]], acc);
  acc = warp_sum_b(acc);
  if (lane == 0) X[L.off + L.gmap[i]] = (T)acc;
}

// ---- solve control (all members of the plan) ----
// start: hist[0] = ||r_0||; members with a zero or non-finite residual, or maxit <= 0, stop here
__global__ void kb_start_check(const double* __restrict__ rr0, int* __restrict__ active, int* __restrict__ it,
                               int* __restrict__ status, double* __restrict__ hist, int cap, const int* __restrict__ ctrl,
                               int n, cudaGraphConditionalHandle hw) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int maxit = ctrl[0];
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const double r0 = sqrt(rr0[g]);
    hist[(long long)g * (cap + 1)] = r0;
    it[g] = 0;
    int st = ST_RUNNING, a = 1;
    if (!isfinite(r0)) { st = ST_NAN; a = 0; }
    else if (r0 == 0.0) { st = ST_CONVERGED; a = 0; }
    else if (maxit <= 0) { st = ST_MAXIT; a = 0; }
    status[g] = st;
    active[g] = a;
    if (a) any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(hw, any);
}
__global__ void kb_step_check(const double* __restrict__ rr, const double* __restrict__ rr0, int* __restrict__ active,
                              int* __restrict__ it, int* __restrict__ status, double* __restrict__ hist, int cap,
                              const int* __restrict__ ctrl, const double* __restrict__ rtol, int n,
                              cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hi, int has_if) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int maxit = ctrl[0];
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    if (!active[g]) continue;
    const int k = ++it[g];
    const double r = sqrt(rr[g]);
    if (k <= cap) hist[(long long)g * (cap + 1) + k] = r;
    if (!isfinite(r)) { status[g] = ST_NAN; active[g] = 0; }
    else if (r <= rtol[0] * sqrt(rr0[g])) { status[g] = ST_CONVERGED; active[g] = 0; }
    else if (k >= maxit) { status[g] = ST_MAXIT; active[g] = 0; }
    else any = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cudaGraphSetConditional(hw, any);
    if (has_if) cudaGraphSetConditional(hi, any);
  }
}

// ---- gather of the right-hand sides (boundary entries zero) and scatter of the solutions ----
__global__ void __launch_bounds__(kChunk)
kb_gather(double* __restrict__ dst, const double* const* __restrict__ src, const BLev* __restrict__ lev,
          const int* __restrict__ cmem, const int* __restrict__ gid) {
  const int mem = cmem[blockIdx.x];
  const BLev& L = lev[mem];
  const long long i = (long long)blockIdx.x * kChunk + threadIdx.x;
  const long long j = i - L.off;
  double v = 0.0;
  if (j < L.m.N) {
    const long long I = j % L.m.Nn[0], r = j / L.m.Nn[0], J = r % L.m.Nn[1], K = r / L.m.Nn[1];
    bool bd = I == 0 || I == L.m.Nn[0] - 1 || J == 0 || J == L.m.Nn[1] - 1;
    if (L.m.dim == 3) bd = bd || K == 0 || K == L.m.Nn[2] - 1;
    if (!bd) v = src[gid[mem]][j];
  }
  dst[i] = v;
}
__global__ void __launch_bounds__(kChunk)
kb_scatter(const double* __restrict__ srcv, double* const* __restrict__ dst, const BLev* __restrict__ lev,
           const int* __restrict__ cmem, const int* __restrict__ gid) {
  const int mem = cmem[blockIdx.x];
  const BLev& L = lev[mem];
  const long long i = (long long)blockIdx.x * kChunk + threadIdx.x;
  const long long j = i - L.off;
  if (j < L.m.N) dst[gid[mem]][j] = srcv[i];
}

// solve parameters, and every member active for the prologue (its dot products and the start test)
__global__ void kb_set(int* __restrict__ ctrl, double* __restrict__ rtol_dev, int maxit, double rtol,
                       int* __restrict__ active, int n) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) active[g] = 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctrl[0] = maxit;
    rtol_dev[0] = rtol;
  }
}

long long round_chunk(long long n) { return (n + kChunk - 1) / kChunk * kChunk; }

}  // namespace

// ----------------------------------------------------------------------------------- plan
struct BGroup {
  int dim = 0, nlev = 0, prec = 0, smoother = 0, nu_pre = 0, nu_post = 0;
  bool mixed = false, flexible = false;
  bool df64 = false;               // finest FP64 operator in double-float arithmetic
  int2* d_tdf = nullptr;           // its work table (member, group of elements), level 0
  int n_tdf = 0;
  std::vector<int> gids;           // plan-wide ids of the members
  std::vector<int> orders;         // per level
  int* d_gid = nullptr;
  // per level
  std::vector<BLev*> d_lev;
  std::vector<long long> len;      // super-vector length (chunks * kChunk)
  std::vector<int*> d_cmem;
  std::vector<int> nchunk;
  std::vector<int2*> d_t64;        // FP64 apply (member, first element)
  std::vector<int> n_t64;
  std::vector<int> v64;            // FP64 apply block shape per level (0..3)
  std::vector<int2*> d_tlow;       // reduced apply (member, group of elements)
  std::vector<int> n_tlow;
  std::vector<void*> vb, vx, vr, vd, vdinv;  // V-cycle vectors (FP32 when mixed, else FP64)
  std::vector<double*> d_inv_theta;
  std::vector<std::vector<double*>> d_c1, d_c2;  // Chebyshev step s >= 1
  double* d_omega = nullptr;
  // transfers between level k and k+1: restrict / prolong passes per axis
  void* t1 = nullptr;
  void* t2 = nullptr;
  std::vector<std::array<BPass*, 3>> d_rp, d_pp;
  std::vector<std::array<int2*, 3>> d_rt, d_pt;
  std::vector<std::array<int, 3>> n_rt, n_pt;
  int2* d_ct = nullptr;            // coarsest GEMV rows
  int n_ct = 0;
  // fine FP64 vectors and the segmented-dot data of level 0
  double *gb = nullptr, *u = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *h = nullptr;
  double* partial = nullptr;
  int* d_cstart = nullptr;
  cudaStream_t cap = nullptr;      // capture stream of this group's branch
};

struct BatchPlan {
  int n = 0, mode = 0, cap = 0, device = 0;
  std::vector<hmg_problem*> probs;
  std::vector<std::unique_ptr<BGroup>> groups;
  std::vector<void*> allocs;
  // plan-wide per-member state
  double *rr0 = nullptr, *rr = nullptr, *rho = nullptr, *ph = nullptr, *beta = nullptr, *rtol = nullptr;
  int *active = nullptr, *it = nullptr, *status = nullptr, *ctrl = nullptr;
  double* hist = nullptr;
  const double** d_src = nullptr;   // per-call pointer tables
  double** d_dst = nullptr;
  // pinned host mirrors
  int* h_it = nullptr;
  int* h_status = nullptr;
  double* h_hist = nullptr;
  void* h_ptrs = nullptr;           // 2n pointers
  cudaStream_t s = nullptr;         // capture / build stream
  cudaGraphExec_t exec = nullptr;
  long long kern[3] = {0, 0, 0};    // kernel nodes: prologue, loop body part 1, part 2
  int* err = nullptr;
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (s) cudaStreamSynchronize(s);
    for (auto& g : groups)
      if (g->cap) cudaStreamDestroy(g->cap);
    for (void* a : allocs) dev_free(a, s);
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    pinned_free(h_it, (size_t)n * sizeof(int));
    pinned_free(h_status, (size_t)n * sizeof(int));
    pinned_free(h_hist, (size_t)n * (cap + 1) * sizeof(double));
    pinned_free(h_ptrs, (size_t)2 * n * sizeof(void*));
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    *p = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = dev_alloc((void**)p, bytes, s);
    if (e != cudaSuccess) return e;
    allocs.push_back((void*)*p);
    return cudaMemsetAsync(*p, 0, bytes, s);
  }
  template <typename T>
  cudaError_t upload(T** p, const std::vector<T>& v) {
    cudaError_t e = alloc(p, v.size());
    if (e != cudaSuccess || v.empty()) return e;
    e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);  // v is a host temporary
  }
};

}  // namespace hmg

using namespace hmg;

#define BTRY(expr)                                                          \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess) {                                                \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));        \
      return _e == cudaErrorMemoryAllocation ? HMG_ENOMEM : HMG_EDEVICE;    \
    }                                                                       \
  } while (0)
#define BCHECK(expr)              \
  do {                            \
    hmg_status _s = (expr);       \
    if (_s != HMG_OK) return _s;  \
  } while (0)

namespace {

// ---- launches of one group (enqueued on stream s, captured into the plan's graph) ----
struct GroupRun {
  BatchPlan& B;
  BGroup& G;
  cudaStream_t s;
  const hmg_desc& D;  // the first member's descriptor (the group shares the smoother settings)

  hmg_status apply_df64(const double* x, double* y, double alpha) {
    if (G.n_tdf == 0) return HMG_OK;
    Basis1D basis;
    make_basis(G.orders[0], &basis);
    auto go = [&](auto nc, auto dc) -> cudaError_t {
      constexpr int N = decltype(nc)::value, DIM = decltype(dc)::value;
      using C = PencilCfg<DIM, N, df64>;
      auto kern = kb_apply_df64<DIM, N>;
      cudaError_t e2 = ensure_smem(kern, C::SMEM);
      if (e2 != cudaSuccess) return e2;
      kern<<<G.n_tdf, C::THREADS, C::SMEM, s>>>(x, y, G.d_lev[0], G.d_tdf, G.d_gid, B.active,
                                                 make_pencil_tab<N, df64>(basis), df64(alpha));
      return counted(cudaGetLastError());
    };
    auto by_dim = [&](auto nc) -> cudaError_t {
      return G.dim == 3 ? go(nc, std::integral_constant<int, 3>{}) : go(nc, std::integral_constant<int, 2>{});
    };
    static_assert(kDf64MaxN == 9, "the dispatch below covers N = 2..9");
    cudaError_t e = cudaErrorInvalidValue;
    switch (basis.n) {
      case 2: e = by_dim(std::integral_constant<int, 2>{}); break;
      case 3: e = by_dim(std::integral_constant<int, 3>{}); break;
      case 4: e = by_dim(std::integral_constant<int, 4>{}); break;
      case 5: e = by_dim(std::integral_constant<int, 5>{}); break;
      case 6: e = by_dim(std::integral_constant<int, 6>{}); break;
      case 7: e = by_dim(std::integral_constant<int, 7>{}); break;
      case 8: e = by_dim(std::integral_constant<int, 8>{}); break;
      case 9: e = by_dim(std::integral_constant<int, 9>{}); break;
      default: break;
    }
    BTRY(e);
    return HMG_OK;
  }
  hmg_status apply64(int k, const double* x, double* y, double alpha) {
    if (k == 0 && G.df64) return apply_df64(x, y, alpha);
    const int n = G.n_t64[k];
    if (n == 0) return HMG_OK;
    const int dim = G.dim, v = G.v64[k];
    Basis1D basis;
    make_basis(G.orders[k], &basis);
    cudaError_t e = dispatch_n(basis.n, [&](auto nc) -> cudaError_t {
      constexpr int N = decltype(nc)::value;
      auto go = [&](auto vc, auto dc) -> cudaError_t {
        constexpr int V = decltype(vc)::value, DIM = decltype(dc)::value;
        using C = Apply64Cfg<DIM, N, V>;
        auto kern = kb_apply64<DIM, N, V>;
        cudaError_t e2 = ensure_smem(kern, C::smem);
        if (e2 != cudaSuccess) return e2;
        kern<<<n, C::GT, C::smem, s>>>(x, y, G.d_lev[k], G.d_t64[k], G.d_gid, B.active, make_tab<N, double>(basis),
                                       alpha, alpha_mode(alpha), B.err);
        return counted(cudaGetLastError());
      };
      auto by_v = [&](auto dc) -> cudaError_t {
        (void)v;
        return go(std::integral_constant<int, 0>{}, dc);
      };
      return dim == 3 ? by_v(std::integral_constant<int, 3>{}) : by_v(std::integral_constant<int, 2>{});
    });
    BTRY(e);
    return HMG_OK;
  }
  hmg_status apply_low(int k, const float* x, float* y, float alpha) {
    const int n = G.n_tlow[k];
    if (n == 0) return HMG_OK;
    Basis1D basis;
    make_basis(G.orders[k], &basis);
    cudaError_t e = dispatch_n(basis.n, [&](auto nc) -> cudaError_t {
      constexpr int N = decltype(nc)::value;
      auto go = [&](auto dc, auto gt) -> cudaError_t {
        constexpr int DIM = decltype(dc)::value;
        using GT = typename decltype(gt)::type;
        using C = PencilCfg<DIM, N>;
        auto kern = kb_apply_low<DIM, N, GT>;
        cudaError_t e2 = ensure_smem(kern, C::SMEM);
        if (e2 != cudaSuccess) return e2;
        kern<<<n, C::THREADS, C::SMEM, s>>>(x, y, G.d_lev[k], G.d_tlow[k], G.d_gid, B.active,
                                            make_pencil_tab<N, float>(basis), alpha);
        return counted(cudaGetLastError());
      };
      auto by_prec = [&](auto dc) -> cudaError_t {
        if (G.prec == HMG_PREC_FP16) return go(dc, std::common_type<__half>{});
        if (G.prec == HMG_PREC_BF16) return go(dc, std::common_type<__nv_bfloat16>{});
        return go(dc, std::common_type<float>{});
      };
      return G.dim == 3 ? by_prec(std::integral_constant<int, 3>{}) : by_prec(std::integral_constant<int, 2>{});
    });
    BTRY(e);
    return HMG_OK;
  }
  hmg_status apply(int k, const double* x, double* y, double alpha) { return apply64(k, x, y, alpha); }
  hmg_status apply(int k, const float* x, float* y, float alpha) { return apply_low(k, x, y, alpha); }

  template <typename T>
  hmg_status vec(int k, void* const* arr, T** out) {
    *out = static_cast<T*>(arr[k]);
    return HMG_OK;
  }

  // `steps` smoothing steps on level k (the batched form of smooth() in hmg.cu)
  template <typename T>
  hmg_status smooth(int k, const T* b, T* x, int steps, bool zero, bool leave_r_b) {
    T* r = static_cast<T*>(G.vr[k]);
    T* d = static_cast<T*>(G.vd[k]);
    const T* dinv = static_cast<const T*>(G.vdinv[k]);
    const long long len = G.len[k];
    const int nc = G.nchunk[k];
    if (steps <= 0) {
      if (zero) BTRY(cudaMemsetAsync(x, 0, len * sizeof(T), s));
      if (leave_r_b) BTRY(cudaMemcpyAsync(r, b, len * sizeof(T), cudaMemcpyDeviceToDevice, s));
      return HMG_OK;
    }
    bool r_is_b = false;
    auto residual = [&]() -> hmg_status {
      if (!r_is_b) BTRY(cudaMemcpyAsync(r, b, len * sizeof(T), cudaMemcpyDeviceToDevice, s));
      return apply(k, x, r, (T)-1);
    };
    if (G.smoother == HMG_SMOOTH_JACOBI || G.smoother == HMG_SMOOTH_L1JACOBI) {
      for (int st = 0; st < steps; ++st) {
        const bool reset = st + 1 < steps || leave_r_b;
        if (st == 0 && zero) {
          kb_jacobi_first<T><<<nc, kChunk, 0, s>>>(x, b, dinv, reset ? r : nullptr, G.d_omega, G.d_cmem[k], G.d_gid,
                                                   B.active);
          BTRY(counted(cudaGetLastError()));
        } else {
          BCHECK(residual());
          kb_jacobi<T><<<nc, kChunk, 0, s>>>(x, r, b, dinv, G.d_omega, reset ? 1 : 0, G.d_cmem[k], G.d_gid, B.active);
          BTRY(counted(cudaGetLastError()));
        }
        r_is_b = reset;
      }
      return HMG_OK;
    }
    for (int st = 0; st < steps; ++st) {  // Chebyshev (Saad, Iterative Methods, Alg. 12.1)
      const bool reset = st + 1 < steps || leave_r_b;
      if (st == 0) {
        if (zero) {
          kb_cheb_first<T><<<nc, kChunk, 0, s>>>(x, d, b, dinv, reset ? r : nullptr, G.d_inv_theta[k], G.d_cmem[k],
                                                 G.d_gid, B.active);
          BTRY(counted(cudaGetLastError()));
        } else {
          BCHECK(residual());
          // the first step from a nonzero guess: c1 = 0, c2 = 1 / theta (the c1[0] / c2[0] tables)
          kb_cheb<T><<<nc, kChunk, 0, s>>>(x, d, r, b, dinv, G.d_c1[k][0], G.d_c2[k][0], reset ? 1 : 0, G.d_cmem[k],
                                           G.d_gid, B.active);
          BTRY(counted(cudaGetLastError()));
        }
      } else {
        BCHECK(residual());
        kb_cheb<T><<<nc, kChunk, 0, s>>>(x, d, r, b, dinv, G.d_c1[k][st], G.d_c2[k][st], reset ? 1 : 0, G.d_cmem[k],
                                         G.d_gid, B.active);
        BTRY(counted(cudaGetLastError()));
      }
      r_is_b = reset;
    }
    return HMG_OK;
  }

  template <typename T>
  hmg_status transfer(int k, bool restrict_dir, const T* in0, T* outl) {
    const auto& passes = restrict_dir ? G.d_rp[k] : G.d_pp[k];
    const auto& tabs = restrict_dir ? G.d_rt[k] : G.d_pt[k];
    const auto& ns = restrict_dir ? G.n_rt[k] : G.n_pt[k];
    T* bufs[2] = {static_cast<T*>(G.t1), static_cast<T*>(G.t2)};
    const T* in = in0;
    for (int a = 0; a < G.dim; ++a) {
      const bool last = a == G.dim - 1;
      T* out = last ? outl : bufs[a & 1];
      if (ns[a] > 0) {
        if (std::is_same<T, float>::value)
          kb_axis<T, float><<<ns[a], kChunk, 0, s>>>(in, out, passes[a], tabs[a], a == 0, last,
                                                      (!restrict_dir && last) ? 1 : 0, G.d_gid, B.active);
        else
          kb_axis<T, double><<<ns[a], kChunk, 0, s>>>(in, out, passes[a], tabs[a], a == 0, last,
                                                       (!restrict_dir && last) ? 1 : 0, G.d_gid, B.active);
        BTRY(counted(cudaGetLastError()));
      }
      in = out;
    }
    return HMG_OK;
  }

  template <typename T>
  hmg_status vcycle(int k, const T* b, T* x, bool zero) {
    const int last = G.nlev - 1;
    if (k == last) {
      BTRY(cudaMemsetAsync(x, 0, G.len[k] * sizeof(T), s));
      if (G.n_ct > 0) {
        kb_coarse<T><<<G.n_ct, 256, 0, s>>>(b, x, G.d_lev[k], G.d_ct, G.d_gid, B.active);
        BTRY(counted(cudaGetLastError()));
      }
      return HMG_OK;
    }
    T* r = static_cast<T*>(G.vr[k]);
    BCHECK(smooth<T>(k, b, x, D.nu_pre, zero, true));  // leaves r = b
    BCHECK(apply(k, x, r, (T)-1));
    BCHECK(transfer<T>(k, true, r, static_cast<T*>(G.vb[k + 1])));
    BCHECK(vcycle<T>(k + 1, static_cast<T*>(G.vb[k + 1]), static_cast<T*>(G.vx[k + 1]), true));
    BCHECK(transfer<T>(k, false, static_cast<T*>(G.vx[k + 1]), x));
    BCHECK(smooth<T>(k, b, x, D.nu_post, false, false));
    return HMG_OK;
  }

  // z = B r on the finest level (FP64 in and out)
  hmg_status precondition(const double* r, double* z) {
    if (G.mixed && G.nlev > 1) {
      float* b32 = static_cast<float*>(G.vb[0]);
      float* x32 = static_cast<float*>(G.vx[0]);
      BTRY(to_f32(b32, r, G.len[0], s));
      BCHECK(vcycle<float>(0, b32, x32, true));
      BTRY(to_f64(z, x32, G.len[0], s));
      return HMG_OK;
    }
    if (G.mixed) {  // a single level: the coarsest solve in the V-cycle precision
      float* b32 = static_cast<float*>(G.vb[0]);
      float* x32 = static_cast<float*>(G.vx[0]);
      BTRY(to_f32(b32, r, G.len[0], s));
      BCHECK(vcycle<float>(0, b32, x32, true));
      BTRY(to_f64(z, x32, G.len[0], s));
      return HMG_OK;
    }
    return vcycle<double>(0, r, z, true);
  }

  hmg_status dot(const double* x, const double* y, int op, double* out, double* aux) {
    kb_dot<double><<<G.nchunk[0], kChunk, 0, s>>>(x, y, G.partial, G.d_cmem[0], G.d_gid, B.active);
    BTRY(counted(cudaGetLastError()));
    const int nm = (int)G.gids.size();
    kb_seg_finish<<<(nm + 127) / 128, 128, 0, s>>>(G.partial, G.d_cstart, nm, G.d_gid, B.active, op, out, aux);
    BTRY(counted(cudaGetLastError()));
    return HMG_OK;
  }

  // prologue: r = b (masked, already in gb), u = 0, rr0
  hmg_status prologue_a() {
    BTRY(cudaMemcpyAsync(G.r, G.gb, G.len[0] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BTRY(cudaMemsetAsync(G.u, 0, G.len[0] * sizeof(double), s));
    return dot(G.r, G.r, SEG_STORE, B.rr0, nullptr);
  }
  // prologue after the start check (PCG): z = V(r), p = z, rho = (z, r)
  hmg_status prologue_b() {
    BCHECK(precondition(G.r, G.z));
    BTRY(cudaMemcpyAsync(G.p, G.z, G.len[0] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return dot(G.z, G.r, SEG_STORE, B.rho, nullptr);
  }
  // PCG part 1: h = A p, alpha, u, r, ||r||^2
  hmg_status pcg_a() {
    BTRY(cudaMemsetAsync(G.h, 0, G.len[0] * sizeof(double), s));
    BCHECK(apply64(0, G.p, G.h, 1.0));
    BCHECK(dot(G.p, G.h, SEG_STORE, B.ph, nullptr));
    kb_pcg_update<<<G.nchunk[0], kChunk, 0, s>>>(G.u, G.r, G.p, G.h, B.rho, B.ph, G.partial, G.d_cmem[0], G.d_gid,
                                                  B.active);
    BTRY(counted(cudaGetLastError()));
    const int nm = (int)G.gids.size();
    kb_seg_finish<<<(nm + 127) / 128, 128, 0, s>>>(G.partial, G.d_cstart, nm, G.d_gid, B.active, SEG_STORE, B.rr,
                                                   nullptr);
    BTRY(counted(cudaGetLastError()));
    return HMG_OK;
  }
  // PCG part 2: z = V(r), rho and beta (flexible for 16-bit V-cycles), p = z + beta p
  hmg_status pcg_b() {
    BCHECK(precondition(G.r, G.z));
    if (G.flexible) {
      BCHECK(dot(G.z, G.h, SEG_NEG_RATIO, B.beta, B.ph));
      BCHECK(dot(G.z, G.r, SEG_STORE, B.rho, nullptr));
    } else {
      BCHECK(dot(G.z, G.r, SEG_RHO_BETA, B.rho, B.beta));
    }
    kb_pcg_dir<<<G.nchunk[0], kChunk, 0, s>>>(G.p, G.z, B.beta, G.d_cmem[0], G.d_gid, B.active);
    BTRY(counted(cudaGetLastError()));
    return HMG_OK;
  }
  // MG iteration: u += V(b - A u) (r holds b - A u), then r = b - A u, ||r||^2
  hmg_status mg_step() {
    BCHECK(precondition(G.r, G.z));
    kb_axpy<<<G.nchunk[0], kChunk, 0, s>>>(G.u, G.z, G.d_cmem[0], G.d_gid, B.active);
    BTRY(counted(cudaGetLastError()));
    BTRY(cudaMemcpyAsync(G.r, G.gb, G.len[0] * sizeof(double), cudaMemcpyDeviceToDevice, s));
    BCHECK(apply64(0, G.u, G.r, -1.0));
    return dot(G.r, G.r, SEG_STORE, B.rr, nullptr);
  }
};

// Fork the plan's capture stream into one branch per group, run fn(group run) on each branch,
// and join back.
template <typename F>
hmg_status for_groups(BatchPlan& B, F&& fn) {
  std::vector<cudaEvent_t> evs;
  auto cleanup = [&]() {
    for (auto e : evs) cudaEventDestroy(e);
  };
  cudaEvent_t fork;
  BTRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  evs.push_back(fork);
  cudaError_t e = cudaEventRecord(fork, B.s);
  if (e != cudaSuccess) { cleanup(); BTRY(e); }
  for (auto& g : B.groups) {
    e = cudaStreamWaitEvent(g->cap, fork, 0);
    if (e != cudaSuccess) { cleanup(); BTRY(e); }
    const hmg_desc& D = B.probs[g->gids[0]]->impl.desc;
    GroupRun run{B, *g, g->cap, D};
    hmg_status st = fn(run);
    if (st != HMG_OK) { cleanup(); return st; }
    cudaEvent_t join;
    e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (e != cudaSuccess) { cleanup(); BTRY(e); }
    evs.push_back(join);
    e = cudaEventRecord(join, g->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B.s, join, 0);
    if (e != cudaSuccess) { cleanup(); BTRY(e); }
  }
  cleanup();
  return HMG_OK;
}

template <typename F>
hmg_status capture_to(cudaGraph_t g, cudaStream_t s, F&& fn, std::vector<cudaGraphNode_t>* leaves) {
  BTRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  hmg_status st = fn();
  if (st == HMG_OK && leaves) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &d, nullptr, &nd);
    if (e == cudaSuccess) leaves->assign(d, d + nd);
    else st = HMG_EDEVICE;
  }
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &out);
  if (st != HMG_OK) return st;
  BTRY(e);
  return HMG_OK;
}

hmg_status add_cond(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h,
                    cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  BTRY(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &prm));
  *body = prm.conditional.phGraph_out[0];
  return HMG_OK;
}

// Signature of a hierarchy's structure: members of one group share it.
std::vector<long long> signature(const ProblemImpl& P) {
  const hmg_desc& D = P.desc;
  std::vector<long long> s = {D.dim, (long long)P.L.size(), D.smoother, D.nu_pre, D.nu_post, D.smooth_prec,
                              (long long)(P.L[0].v64 == kApply64Df)};
  for (const Level& l : P.L) s.push_back(l.m.p);
  return s;
}

hmg_status build_group(BatchPlan& B, BGroup& G) {
  const ProblemImpl& P0 = B.probs[G.gids[0]]->impl;
  const hmg_desc& D0 = P0.desc;
  G.dim = D0.dim;
  G.nlev = (int)P0.L.size();
  G.prec = D0.smooth_prec;
  G.mixed = D0.smooth_prec != HMG_PREC_FP64;
  G.flexible = D0.smooth_prec == HMG_PREC_FP16 || D0.smooth_prec == HMG_PREC_BF16;
  G.df64 = P0.L[0].v64 == kApply64Df;
  G.smoother = D0.smoother;
  G.nu_pre = D0.nu_pre;
  G.nu_post = D0.nu_post;
  for (const Level& l : P0.L) G.orders.push_back(l.m.p);
  const int nm = (int)G.gids.size();
  const size_t vsz = G.mixed ? sizeof(float) : sizeof(double);
  BTRY(B.upload(&G.d_gid, G.gids));
  std::vector<std::vector<long long>> off(G.nlev, std::vector<long long>(nm));
  G.d_lev.resize(G.nlev);
  G.len.resize(G.nlev);
  G.d_cmem.resize(G.nlev);
  G.nchunk.resize(G.nlev);
  G.d_t64.resize(G.nlev);
  G.n_t64.resize(G.nlev);
  G.v64.resize(G.nlev);
  G.d_tlow.resize(G.nlev);
  G.n_tlow.resize(G.nlev);
  G.vb.resize(G.nlev);
  G.vx.resize(G.nlev);
  G.vr.resize(G.nlev);
  G.vd.resize(G.nlev);
  G.vdinv.resize(G.nlev);
  G.d_inv_theta.resize(G.nlev);
  G.d_c1.resize(G.nlev);
  G.d_c2.resize(G.nlev);
  const int maxnu = std::max(std::max(D0.nu_pre, D0.nu_post), 1);
  std::vector<double> omega(nm);
  for (int m = 0; m < nm; ++m) omega[m] = B.probs[G.gids[m]]->impl.desc.omega;
  BTRY(B.upload(&G.d_omega, omega));
  for (int k = 0; k < G.nlev; ++k) {
    std::vector<BLev> lev(nm);
    std::vector<int> cmem;
    std::vector<int2> t64, tlow, tdf;
    long long o = 0;
    // the FP64 apply of a group: block shape 0 (about one warp of whole elements per block), which
    // suits the small meshes batches are made of
    G.v64[k] = 0;
    const int n1 = G.orders[k] + 1;
    const long long np = G.dim == 3 ? (long long)n1 * n1 * n1 : (long long)n1 * n1;
    const int neg = apply64_neg((int)np, G.v64[k]);
    const int epb = pencil_shape(G.dim, n1).epb;
    for (int m = 0; m < nm; ++m) {
      const Level& l = B.probs[G.gids[m]]->impl.L[k];
      off[k][m] = o;
      BLev& L = lev[m];
      L.m = l.m;
      L.off = o;
      L.G = l.G;
      L.Glow = l.Glow;
      L.Gdf = l.Gdf;
      L.gsc = l.gsc;
      L.Ainv = l.Ainv;
      L.gmap = l.gmap;
      L.nI = l.Ainv ? l.nI : 0;
      const long long seg = round_chunk(l.m.N);
      for (long long c = 0; c < seg / kChunk; ++c) cmem.push_back(m);
      for (long long e = 0; e < l.m.nelem; e += neg) t64.push_back(make_int2(m, (int)e));
      if (G.mixed)
        for (long long g = 0; g * epb < l.m.nelem; ++g) tlow.push_back(make_int2(m, (int)g));
      if (k == 0 && G.df64)  // the double-float pencil form groups elements as the FP32 one does
        for (long long g = 0; g * epb < l.m.nelem; ++g) tdf.push_back(make_int2(m, (int)g));
      o += seg;
    }
    G.len[k] = o;
    G.nchunk[k] = (int)cmem.size();
    BTRY(B.upload(&G.d_lev[k], lev));
    BTRY(B.upload(&G.d_cmem[k], cmem));
    const bool need64 = !G.mixed || k == 0;
    G.n_t64[k] = need64 ? (int)t64.size() : 0;
    if (need64) BTRY(B.upload(&G.d_t64[k], t64));
    G.n_tlow[k] = G.mixed ? (int)tlow.size() : 0;
    if (G.mixed) BTRY(B.upload(&G.d_tlow[k], tlow));
    if (k == 0 && G.df64) {
      G.n_tdf = (int)tdf.size();
      BTRY(B.upload(&G.d_tdf, tdf));
    }
    // V-cycle vectors and the smoother's inverse diagonal, in the V-cycle precision
    void** vs[4] = {&G.vb[k], &G.vx[k], &G.vr[k], &G.vd[k]};
    for (void** v : vs) BTRY(B.alloc((unsigned char**)v, (size_t)o * vsz));
    BTRY(B.alloc((unsigned char**)&G.vdinv[k], (size_t)o * vsz));
    for (int m = 0; m < nm; ++m) {
      const Level& l = B.probs[G.gids[m]]->impl.L[k];
      const void* src = G.mixed ? (const void*)l.dinv32 : (const void*)l.dinv;
      if (src)
        BTRY(cudaMemcpyAsync(static_cast<unsigned char*>(G.vdinv[k]) + off[k][m] * vsz, src, (size_t)l.m.N * vsz,
                             cudaMemcpyDeviceToDevice, B.s));
    }
    // Chebyshev coefficients per member (the recurrence of smooth() in hmg.cu)
    if (k + 1 < G.nlev && G.smoother == HMG_SMOOTH_CHEB) {
      std::vector<double> inv_theta(nm);
      std::vector<std::vector<double>> c1(maxnu, std::vector<double>(nm)), c2(maxnu, std::vector<double>(nm));
      for (int m = 0; m < nm; ++m) {
        const ProblemImpl& P = B.probs[G.gids[m]]->impl;
        const double hi = P.desc.cheb_safety * P.L[k].lam, lo = P.desc.cheb_lo_frac * hi;
        const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
        const double sigma = theta / delta;
        double rho = 1.0 / sigma;
        inv_theta[m] = 1.0 / theta;
        c1[0][m] = 0.0;
        c2[0][m] = 1.0 / theta;
        for (int st = 1; st < maxnu; ++st) {
          const double rho_new = 1.0 / (2.0 * sigma - rho);
          c1[st][m] = rho_new * rho;
          c2[st][m] = 2.0 * rho_new / delta;
          rho = rho_new;
        }
      }
      BTRY(B.upload(&G.d_inv_theta[k], inv_theta));
      G.d_c1[k].resize(maxnu);
      G.d_c2[k].resize(maxnu);
      for (int st = 0; st < maxnu; ++st) {
        BTRY(B.upload(&G.d_c1[k][st], c1[st]));
        BTRY(B.upload(&G.d_c2[k][st], c2[st]));
      }
    }
  }
  // transfers: per member, scratch for the intermediate passes of both directions
  std::vector<long long> toff(nm);
  long long tlen = 0;
  for (int m = 0; m < nm; ++m) {
    const ProblemImpl& P = B.probs[G.gids[m]]->impl;
    long long need = 0;
    for (int k = 0; k + 1 < G.nlev; ++k) {
      const Mesh& f = P.L[k].m;
      const Mesh& c = P.L[k + 1].m;
      long long od[3] = {f.Nn[0], f.Nn[1], f.Nn[2]};
      for (int a = 0; a + 1 < G.dim; ++a) {
        od[a] = c.Nn[a];
        need = std::max(need, od[0] * od[1] * od[2]);
      }
      long long op[3] = {c.Nn[0], c.Nn[1], c.Nn[2]};
      for (int a = 0; a + 1 < G.dim; ++a) {
        op[a] = f.Nn[a];
        need = std::max(need, op[0] * op[1] * op[2]);
      }
    }
    toff[m] = tlen;
    tlen += round_chunk(std::max(1LL, need));
  }
  BTRY(B.alloc((unsigned char**)&G.t1, (size_t)tlen * vsz));
  BTRY(B.alloc((unsigned char**)&G.t2, (size_t)tlen * vsz));
  const int npair = std::max(0, G.nlev - 1);
  G.d_rp.resize(npair);
  G.d_pp.resize(npair);
  G.d_rt.resize(npair);
  G.d_pt.resize(npair);
  G.n_rt.resize(npair);
  G.n_pt.resize(npair);
  for (int k = 0; k < npair; ++k) {
    for (int dir = 0; dir < 2; ++dir) {  // 0 restrict (fine -> coarse), 1 prolong (coarse -> fine)
      for (int a = 0; a < G.dim; ++a) {
        std::vector<BPass> ps(nm);
        std::vector<int2> tab;
        for (int m = 0; m < nm; ++m) {
          const ProblemImpl& P = B.probs[G.gids[m]]->impl;
          const Level& fl = P.L[k];
          const Mesh& f = fl.m;
          const Mesh& c = P.L[k + 1].m;
          long long od[3];
          for (int q = 0; q < 3; ++q) od[q] = dir == 0 ? f.Nn[q] : c.Nn[q];
          for (int q = 0; q <= a; ++q) od[q] = dir == 0 ? c.Nn[q] : f.Nn[q];
          BPass& bp = ps[m];
          const bool last = a == G.dim - 1;
          bp.in_off = a == 0 ? off[dir == 0 ? k : k + 1][m] : toff[m];
          bp.out_off = last ? off[dir == 0 ? k + 1 : k][m] : toff[m];
          for (int q = 0; q < 3; ++q) bp.od[q] = od[q];
          bp.axis = a;
          const Axis1D& ax = dir == 0 ? fl.PT[a] : fl.P[a];
          bp.n_in = ax.n_in;
          bp.rowptr = ax.rowptr;
          bp.col = ax.col;
          bp.val = ax.val;
          bp.val32 = ax.val32;
          const long long tot = od[0] * od[1] * od[2];
          for (long long t0 = 0; t0 < tot; t0 += kChunk) tab.push_back(make_int2(m, (int)t0));
        }
        BPass* dp = nullptr;
        int2* dt = nullptr;
        BTRY(B.upload(&dp, ps));
        BTRY(B.upload(&dt, tab));
        (dir == 0 ? G.d_rp : G.d_pp)[k][a] = dp;
        (dir == 0 ? G.d_rt : G.d_pt)[k][a] = dt;
        (dir == 0 ? G.n_rt : G.n_pt)[k][a] = (int)tab.size();
      }
    }
  }
  // coarsest GEMV rows (8 per block)
  {
    std::vector<int2> ct;
    for (int m = 0; m < nm; ++m) {
      const Level& l = B.probs[G.gids[m]]->impl.L[G.nlev - 1];
      if (!l.Ainv) continue;
      for (long long i = 0; i < l.nI; i += 8) ct.push_back(make_int2(m, (int)i));
    }
    G.n_ct = (int)ct.size();
    BTRY(B.upload(&G.d_ct, ct));
  }
  // fine FP64 vectors and segmented-dot tables
  const long long n0 = G.len[0];
  double** fv[6] = {&G.gb, &G.u, &G.r, &G.z, &G.p, &G.h};
  for (double** v : fv) BTRY(B.alloc(v, (size_t)n0));
  BTRY(B.alloc(&G.partial, (size_t)G.nchunk[0]));
  std::vector<int> cstart(nm + 1);
  for (int m = 0; m < nm; ++m) cstart[m] = (int)(off[0][m] / kChunk);
  cstart[nm] = G.nchunk[0];
  BTRY(B.upload(&G.d_cstart, cstart));
  BTRY(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
  return HMG_OK;
}

hmg_status build_graph(BatchPlan& B) {
  cudaGraph_t g = nullptr;
  BTRY(cudaGraphCreate(&g, 0));
  hmg_status st = [&]() -> hmg_status {
    cudaGraphConditionalHandle hw;
    BTRY(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
    std::vector<cudaGraphNode_t> leaves;
    long long c0 = add_launches(0);
    BCHECK(capture_to(g, B.s, [&]() -> hmg_status {
      BCHECK(for_groups(B, [&](GroupRun& R) { return R.prologue_a(); }));
      kb_start_check<<<1, 1024, 0, B.s>>>(B.rr0, B.active, B.it, B.status, B.hist, B.cap, B.ctrl, B.n, hw);
      BTRY(counted(cudaGetLastError()));
      if (B.mode == HMG_MODE_PCG) BCHECK(for_groups(B, [&](GroupRun& R) { return R.prologue_b(); }));
      return HMG_OK;
    }, &leaves));
    B.kern[0] = add_launches(0) - c0;
    cudaGraph_t body;
    BCHECK(add_cond(g, leaves, hw, cudaGraphCondTypeWhile, &body));
    c0 = add_launches(0);
    if (B.mode == HMG_MODE_MG) {
      BCHECK(capture_to(body, B.s, [&]() -> hmg_status {
        BCHECK(for_groups(B, [&](GroupRun& R) { return R.mg_step(); }));
        kb_step_check<<<1, 1024, 0, B.s>>>(B.rr, B.rr0, B.active, B.it, B.status, B.hist, B.cap, B.ctrl, B.rtol, B.n,
                                           hw, hw, 0);
        BTRY(counted(cudaGetLastError()));
        return HMG_OK;
      }, nullptr));
      B.kern[1] = add_launches(0) - c0;
    } else {
      cudaGraphConditionalHandle hi;
      BTRY(cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault));
      std::vector<cudaGraphNode_t> l1;
      BCHECK(capture_to(body, B.s, [&]() -> hmg_status {
        BCHECK(for_groups(B, [&](GroupRun& R) { return R.pcg_a(); }));
        kb_step_check<<<1, 1024, 0, B.s>>>(B.rr, B.rr0, B.active, B.it, B.status, B.hist, B.cap, B.ctrl, B.rtol, B.n,
                                           hw, hi, 1);
        BTRY(counted(cudaGetLastError()));
        return HMG_OK;
      }, &l1));
      B.kern[1] = add_launches(0) - c0;
      c0 = add_launches(0);
      cudaGraph_t rest;
      BCHECK(add_cond(body, l1, hi, cudaGraphCondTypeIf, &rest));
      BCHECK(capture_to(rest, B.s, [&]() -> hmg_status {
        return for_groups(B, [&](GroupRun& R) { return R.pcg_b(); });
      }, nullptr));
      B.kern[2] = add_launches(0) - c0;
    }
    add_launches(-(B.kern[0] + B.kern[1] + B.kern[2]));  // captured, not launched
    BTRY(cudaGraphInstantiate(&B.exec, g, 0));
    return HMG_OK;
  }();
  cudaGraphDestroy(g);
  return st;
}

}  // namespace

namespace hmg {

// Whether a problem can join a grouped batch (block-Jacobi smoothing has no grouped form).
bool batch_supported(const hmg_problem* p) {
  return p && !p->impl.L.empty() && p->impl.desc.smoother != HMG_SMOOTH_BLOCKJACOBI;
}

}  // namespace hmg

extern "C" hmg_status hmg_batch_create(hmg_problem* const* probs, int n, int mode, int maxit_cap,
                                       hmg_batch** out) {
  if (!out || !probs || n <= 0 || maxit_cap < 0 || (mode != HMG_MODE_MG && mode != HMG_MODE_PCG)) {
    set_error("hmg_batch_create: bad argument");
    return HMG_EINVAL;
  }
  *out = nullptr;
  int dev = 0;
  BTRY(cudaGetDevice(&dev));
  for (int i = 0; i < n; ++i) {
    if (!batch_supported(probs[i])) {
      set_error("hmg_batch_create: a null handle, or a problem with element-block Jacobi smoothing (no grouped form)");
      return HMG_EINVAL;
    }
    if (probs[i]->impl.device != dev) {
      set_error("hmg_batch_create: every problem must live on the current device");
      return HMG_EINVAL;
    }
    for (int j = 0; j < i; ++j)
      if (probs[j] == probs[i]) { set_error("hmg_batch_create: a handle appears twice"); return HMG_EINVAL; }
  }
  std::unique_ptr<BatchPlan> B(new BatchPlan());
  B->n = n;
  B->mode = mode;
  B->cap = std::max(maxit_cap, 1);
  B->device = dev;
  B->probs.assign(probs, probs + n);
  BTRY(cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking));
  // groups by hierarchy structure, in order of first appearance
  std::vector<std::vector<long long>> sigs;
  for (int i = 0; i < n; ++i) {
    const auto sg = signature(probs[i]->impl);
    size_t gi = 0;
    while (gi < sigs.size() && sigs[gi] != sg) ++gi;
    if (gi == sigs.size()) {
      sigs.push_back(sg);
      B->groups.emplace_back(new BGroup());
    }
    B->groups[gi]->gids.push_back(i);
  }
  BTRY(B->alloc(&B->rr0, n));
  BTRY(B->alloc(&B->rr, n));
  BTRY(B->alloc(&B->rho, n));
  BTRY(B->alloc(&B->ph, n));
  BTRY(B->alloc(&B->beta, n));
  BTRY(B->alloc(&B->rtol, 1));
  BTRY(B->alloc(&B->active, n));
  BTRY(B->alloc(&B->it, n));
  BTRY(B->alloc(&B->status, n));
  BTRY(B->alloc(&B->ctrl, 4));
  BTRY(B->alloc(&B->err, 1));
  BTRY(B->alloc(&B->hist, (size_t)n * (B->cap + 1)));
  BTRY(B->alloc(&B->d_src, n));
  BTRY(B->alloc(&B->d_dst, n));
  B->h_it = static_cast<int*>(pinned_alloc((size_t)n * sizeof(int)));
  B->h_status = static_cast<int*>(pinned_alloc((size_t)n * sizeof(int)));
  B->h_hist = static_cast<double*>(pinned_alloc((size_t)n * (B->cap + 1) * sizeof(double)));
  B->h_ptrs = pinned_alloc((size_t)2 * n * sizeof(void*));
  if (!B->h_it || !B->h_status || !B->h_hist || !B->h_ptrs) {
    set_error("hmg_batch_create: pinned host allocation failed");
    return HMG_ENOMEM;
  }
  for (auto& g : B->groups) BCHECK(build_group(*B, *g));
  BTRY(cudaStreamSynchronize(B->s));
  BCHECK(build_graph(*B));
  *out = reinterpret_cast<hmg_batch*>(B.release());
  return HMG_OK;
}

extern "C" hmg_status hmg_batch_solve(hmg_batch* plan, const double* const* b_dev, double* const* u_dev, double rtol,
                                      int maxit, int* iters, double* const* res_hist, int* status, void* stream) {
  BatchPlan* B = reinterpret_cast<BatchPlan*>(plan);
  if (!B || !b_dev || !u_dev || maxit < 0 || !(rtol >= 0.0)) {
    set_error("hmg_batch_solve: bad argument");
    return HMG_EINVAL;
  }
  if (maxit > B->cap) {
    set_error("hmg_batch_solve: maxit exceeds the plan's capacity");
    return HMG_EINVAL;
  }
  for (int i = 0; i < B->n; ++i)
    if (!b_dev[i] || !u_dev[i]) { set_error("hmg_batch_solve: null vector"); return HMG_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  const int n = B->n;
  const void** hp = static_cast<const void**>(B->h_ptrs);
  for (int i = 0; i < n; ++i) {
    hp[i] = b_dev[i];
    hp[n + i] = u_dev[i];
  }
  BTRY(cudaMemcpyAsync(B->d_src, hp, n * sizeof(void*), cudaMemcpyHostToDevice, s));
  BTRY(cudaMemcpyAsync(B->d_dst, hp + n, n * sizeof(void*), cudaMemcpyHostToDevice, s));
  kb_set<<<(n + 255) / 256, 256, 0, s>>>(B->ctrl, B->rtol, maxit, rtol, B->active, n);
  BTRY(counted(cudaGetLastError()));
  for (auto& g : B->groups) {
    kb_gather<<<g->nchunk[0], kChunk, 0, s>>>(g->gb, B->d_src, g->d_lev[0], g->d_cmem[0], g->d_gid);
    BTRY(counted(cudaGetLastError()));
  }
  BTRY(cudaGraphLaunch(B->exec, s));
  for (auto& g : B->groups) {
    kb_scatter<<<g->nchunk[0], kChunk, 0, s>>>(g->u, B->d_dst, g->d_lev[0], g->d_cmem[0], g->d_gid);
    BTRY(counted(cudaGetLastError()));
  }
  BTRY(cudaMemcpyAsync(B->h_it, B->it, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  BTRY(cudaMemcpyAsync(B->h_status, B->status, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  BTRY(cudaMemcpyAsync(B->h_hist, B->hist, (size_t)n * (B->cap + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  int herr = 0;
  BTRY(cudaMemcpyAsync(&herr, B->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  BTRY(cudaStreamSynchronize(s));
  if (herr) {
    BTRY(cudaMemsetAsync(B->err, 0, sizeof(int), s));
    set_error("a bounded wait inside a kernel gave up (error code " + std::to_string(herr) + ")");
    return HMG_ETIMEOUT;
  }
  int loops = 0;
  hmg_status ret = HMG_OK;
  for (int i = 0; i < n; ++i) {
    const int it = B->h_it[i];
    loops = std::max(loops, it);
    if (iters) iters[i] = it;
    if (res_hist && res_hist[i])
      for (int k = 0; k <= it && k <= B->cap; ++k) res_hist[i][k] = B->h_hist[(size_t)i * (B->cap + 1) + k];
    hmg_status si;
    switch (B->h_status[i]) {
      case ST_CONVERGED: si = HMG_OK; break;
      case ST_MAXIT: si = HMG_ENOCONV; break;
      case ST_NAN: si = HMG_ENAN; break;
      default: si = HMG_EDEVICE; break;
    }
    if (status) status[i] = si;
    if (si != HMG_OK && ret == HMG_OK) ret = si;
    // finest-level applies of this member (cost-model accounting, as for a graph solve)
    ProblemImpl& P = B->probs[i]->impl;
    const hmg_desc& D = P.desc;
    const long long v = P.L.size() < 2 ? 0 : (D.nu_pre >= 1 ? D.nu_pre - 1 : 0) + 1 + D.nu_post;
    if (it > 0) P.fine_applies += B->mode == HMG_MODE_MG ? (long long)it * (v + 1) : v + it + (long long)(it - 1) * v;
    else if (B->mode == HMG_MODE_PCG && B->h_status[i] != ST_NAN) P.fine_applies += v;
  }
  // kernels the graph executed: prologue, one loop body per loop iteration, and (PCG) the second
  // half of every iteration but the last
  add_launches(B->kern[0] + (long long)loops * B->kern[1] + (loops > 0 ? (long long)(loops - 1) * B->kern[2] : 0));
  if (ret == HMG_ENOCONV) set_error("maximum number of iterations reached");
  else if (ret == HMG_ENAN) set_error("non-finite residual");
  return ret;
}

extern "C" hmg_status hmg_batch_destroy(hmg_batch* plan) {
  delete reinterpret_cast<BatchPlan*>(plan);
  return HMG_OK;
}

extern "C" hmg_status hmg_batch_info(const hmg_batch* plan, int* groups, long long* kernels_per_iteration) {
  const BatchPlan* B = reinterpret_cast<const BatchPlan*>(plan);
  if (!B) { set_error("null plan"); return HMG_EINVAL; }
  if (groups) *groups = (int)B->groups.size();
  if (kernels_per_iteration) *kernels_per_iteration = B->kern[1] + B->kern[2];
  return HMG_OK;
}
