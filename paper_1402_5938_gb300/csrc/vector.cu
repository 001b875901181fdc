// Level-vector kernels (see vector.cuh). All loops are grid-stride with a fixed grid so
// that every reduction sums its terms in the same order on every call (deterministic).
#include <math.h>

#include <algorithm>

#include <type_traits>

#include "tma.cuh"
#include "vector.cuh"
#include "ops.cuh"

namespace hmg {

namespace {

constexpr int kThreads = 256;

inline unsigned grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  if (g > (long long)device_sm_count() * 16) g = (long long)device_sm_count() * 16;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

// Blocks of a reduction over n entries: about 4 entries per thread, at most kRedBlocks. Fixed
// for a given n, so sums are reproducible; small vectors use few blocks and leave the GPU to
// other streams' work.
int red_blocks(long long n) {
  long long b = (n + 4LL * kThreads - 1) / (4LL * kThreads);
  if (b < 1) b = 1;
  if (b > kRedBlocks) b = kRedBlocks;
  return (int)b;
}

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (blockDim.x == kThreads); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[kThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < kThreads / 32 ? red[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot_partial(const T* __restrict__ x, const T* __restrict__ y,
                                                          long long n, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    acc = fma((double)x[i], (double)y[i], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_finish(const double* __restrict__ partial, int np, double* S,
                                                     int op, int idx, int aux) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += kThreads) acc += partial[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    if (op == FIN_STORE) S[idx] = acc;
    else if (op == FIN_SQRT) S[idx] = sqrt(acc);
    else if (op == FIN_NEG_RATIO) S[idx] = S[aux] != 0.0 ? -acc / S[aux] : 0.0;
    else {  // FIN_RHO_BETA: beta = new / old, rho = new
      S[aux] = acc / S[idx];
      S[idx] = acc;
    }
  }
}

// Block-Gram-Schmidt helpers (Arnoldi): partial[i * gridDim.x + b] = sum over block b's range
// of V_i . w for the cnt vectors V_i = V + i * ldv (blockIdx.y = i).
__global__ void __launch_bounds__(kThreads) k_multi_dot(const double* __restrict__ V, long long ldv,
                                                        const double* __restrict__ w, long long n,
                                                        double* __restrict__ partial) {
  const double* v = V + blockIdx.y * ldv;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)kThreads + threadIdx.x; t < n; t += (long long)gridDim.x * kThreads)
    acc = fma(v[t], w[t], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// c[i] = sum_b partial[i * np + b] (fixed order); H[i * ldh] += c[i]  (blockIdx.x = i)
__global__ void __launch_bounds__(kThreads) k_multi_finish(const double* __restrict__ partial, int np,
                                                           double* __restrict__ c, double* __restrict__ H,
                                                           int ldh) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < np; b += kThreads) acc += partial[blockIdx.x * np + b];
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    c[blockIdx.x] = acc;
    H[blockIdx.x * ldh] += acc;
  }
}

// w -= sum_{i < cnt} c[i] V_i
__global__ void __launch_bounds__(kThreads) k_multi_axpy(double* __restrict__ w, const double* __restrict__ V,
                                                         long long ldv, int cnt, const double* __restrict__ c,
                                                         long long n) {
  for (long long t = blockIdx.x * (long long)kThreads + threadIdx.x; t < n; t += (long long)gridDim.x * kThreads) {
    double acc = w[t];
    for (int i = 0; i < cnt; ++i) acc = fma(-c[i], V[i * ldv + t], acc);
    w[t] = acc;
  }
}

__global__ void __launch_bounds__(kThreads) k_pcg_update(double* __restrict__ u, double* __restrict__ r,
                                                         const double* __restrict__ p, const double* __restrict__ h,
                                                         long long n, const double* __restrict__ S,
                                                         double* __restrict__ partial) {
  const double ph = S[S_PH];
  const double alpha = ph != 0.0 ? S[S_RHO] / ph : 0.0;  // p = 0 (zero right-hand side): no step
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    u[i] = fma(alpha, p[i], u[i]);
    const double ri = fma(-alpha, h[i], r[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_pcg_dir(double* __restrict__ p, const double* __restrict__ z, long long n,
                          const double* __restrict__ S) {
  const double beta = S[S_BETA];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

template <typename T>
__global__ void k_jacobi_first(T* __restrict__ x, const T* __restrict__ b, const T* __restrict__ dinv, long long n,
                               T omega, T* __restrict__ r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T bi = b[i];
    x[i] = omega * dinv[i] * bi;
    if (r) r[i] = bi;
  }
}

template <typename T>
__global__ void k_jacobi(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ b, const T* __restrict__ dinv,
                         long long n, T omega, int reset) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(omega * dinv[i], r[i], x[i]);
    if (reset) r[i] = b[i];
  }
}

template <typename T>
__global__ void k_cheb_first(T* __restrict__ x, T* __restrict__ d, const T* __restrict__ b,
                             const T* __restrict__ dinv, long long n, T inv_theta, T* __restrict__ r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T bi = b[i];
    const T v = dinv[i] * bi * inv_theta;
    d[i] = v;
    x[i] = v;
    if (r) r[i] = bi;
  }
}

template <typename T>
__global__ void k_cheb(T* __restrict__ x, T* __restrict__ d, T* __restrict__ r, const T* __restrict__ b,
                       const T* __restrict__ dinv, long long n, T c1, T c2, int reset) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T v = fma(c1, d[i], c2 * dinv[i] * r[i]);
    d[i] = v;
    x[i] += v;
    if (reset) r[i] = b[i];
  }
}

__global__ void k_dinv(const double* __restrict__ diag, double* __restrict__ dinv, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dinv[i] = diag[i] != 0.0 ? 1.0 / diag[i] : 0.0;
}

// Probe of one color class for the l1 row norms: v[g] = 1 where g is an interior node whose axis
// indices are congruent to (c0, c1, c2) modulo `period`, else 0.
__global__ void k_color_indicator(double* __restrict__ v, const Mesh m, int period, int c0, int c1, int c2) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < m.N; g += (long long)gridDim.x * blockDim.x) {
    const long long I = g % m.Nn[0];
    const long long r = g / m.Nn[0];
    const long long J = r % m.Nn[1];
    const long long K = m.dim == 3 ? r / m.Nn[1] : 0;
    bool in = I > 0 && I < m.Nn[0] - 1 && J > 0 && J < m.Nn[1] - 1;
    if (m.dim == 3) in = in && K > 0 && K < m.Nn[2] - 1;
    v[g] = (in && I % period == c0 && J % period == c1 && K % period == c2) ? 1.0 : 0.0;
  }
}

__global__ void k_accum_abs(double* __restrict__ acc, const double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc[i] += fabs(y[i]);
}

__device__ __forceinline__ bool on_boundary(long long g, const Mesh& m) {
  const long long I = g % m.Nn[0];
  const long long r = g / m.Nn[0];
  const long long J = r % m.Nn[1];
  const long long K = r / m.Nn[1];
  bool b = (I == 0) | (I == m.Nn[0] - 1) | (J == 0) | (J == m.Nn[1] - 1);
  if (m.dim == 3) b |= (K == 0) | (K == m.Nn[2] - 1);
  return b;
}

__global__ void k_mask(double* __restrict__ v, const Mesh m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m.N; i += (long long)gridDim.x * blockDim.x)
    if (on_boundary(i, m)) v[i] = 0.0;
}

__global__ void k_copy_masked(double* __restrict__ d, const double* __restrict__ s, const Mesh m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m.N; i += (long long)gridDim.x * blockDim.x)
    d[i] = on_boundary(i, m) ? 0.0 : s[i];
}

__global__ void k_to_f32(float* __restrict__ d, const double* __restrict__ s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = (float)s[i];
}

__global__ void k_to_f64(double* __restrict__ d, const float* __restrict__ s, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = (double)s[i];
}

// SplitMix64 (Steele, Lea & Flood 2014), counter form: z = seed + (c+1)*gamma, two
// xor-shift-multiply rounds, final xor-shift; U(-1,1) = 2*(z>>11)*2^-53 - 1.
__global__ void k_start(double* __restrict__ v, const Mesh m, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m.N; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double u = 2.0 * (double)(z >> 11) * 0x1.0p-53 - 1.0;
    v[i] = on_boundary(i, m) ? 0.0 : u;
  }
}

__global__ void k_scale_by(double* __restrict__ w, const double* __restrict__ dinv, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    w[i] *= dinv[i];
}

__global__ void k_axpy_dev(double* __restrict__ y, const double* __restrict__ x, long long n,
                           const double* __restrict__ coef, double sign) {
  const double c = sign * coef[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(c, x[i], y[i]);
}

__global__ void k_div_dev(double* __restrict__ y, const double* __restrict__ x, long long n,
                          const double* __restrict__ den) {
  const double c = den[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] / c;
}

__global__ void k_copy_scalar(double* d, const double* s) { d[0] = s[0]; }

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, long long n, double a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

__global__ void k_set_params(double* S, int* ctrl, double rtol, int maxit, int cap) {
  S[S_RTOL] = rtol;
  ctrl[0] = 0;
  ctrl[1] = ST_RUNNING;
  ctrl[2] = maxit;
  ctrl[3] = cap;
}

__global__ void k_start_check(const double* S, int* ctrl, double* hist, cudaGraphConditionalHandle hw) {
  const double r0 = sqrt(S[S_RR0]);
  hist[0] = r0;
  int cont = 0;
  if (!isfinite(r0)) ctrl[1] = ST_NAN;
  else if (r0 == 0.0) ctrl[1] = ST_CONVERGED;
  else if (ctrl[2] <= 0) ctrl[1] = ST_MAXIT;
  else cont = 1;
  cudaGraphSetConditional(hw, cont);
}

__global__ void k_step_check(const double* S, int* ctrl, double* hist, cudaGraphConditionalHandle hw,
                             cudaGraphConditionalHandle hi, int has_if) {
  const int it = ++ctrl[0];
  const double r = sqrt(S[S_RR]);
  if (it <= ctrl[3]) hist[it] = r;
  int cont = 0;
  if (!isfinite(r)) ctrl[1] = ST_NAN;
  else if (r <= S[S_RTOL] * sqrt(S[S_RR0])) ctrl[1] = ST_CONVERGED;
  else if (it >= ctrl[2]) ctrl[1] = ST_MAXIT;
  else cont = 1;
  cudaGraphSetConditional(hw, cont);
  if (has_if) cudaGraphSetConditional(hi, cont);
}

// Waits on an mbarrier that nothing ever arrives at (no copy in flight), with `polls` polls,
// and records whether the bounded wait gave up: exercises the timeout path the kernels use.
__global__ void k_wait_probe(uint32_t polls, int* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    out[0] = mbar_wait(&bar, 0, polls) ? 0 : 1;
  }
}

struct Gll {
  double r[kMaxN];
};

__global__ void k_node_coords(double* __restrict__ xyz, const Mesh m, const Gll g, double amp) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m.N; t += (long long)gridDim.x * blockDim.x) {
    const long long idx[3] = {t % m.Nn[0], (t / m.Nn[0]) % m.Nn[1], t / (m.Nn[0] * m.Nn[1])};
    double X[3], s = 1.0;
    for (int a = 0; a < m.dim; ++a) {
      const long long e = min(idx[a] / m.p, (long long)m.E[a] - 1);
      X[a] = ((double)e + g.r[idx[a] - e * m.p]) / (double)m.E[a];
      s *= sinpi(X[a]);
    }
    for (int a = 0; a < m.dim; ++a) xyz[a * m.N + t] = X[a] + amp * s;
  }
}

template <typename T, typename V>
__global__ void k_axis(const T* __restrict__ in, T* __restrict__ out, unsigned o0, unsigned o1, unsigned o2,
                       int axis, int n_in, const int* __restrict__ rowptr, const int* __restrict__ col,
                       const V* __restrict__ val, int mask_in, int mask_out, int acc) {
  const unsigned tot = o0 * o1 * o2;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x)
    axis_point<T, V>(in, out, t, o0, o1, o2, axis, n_in, rowptr, col, val, mask_in, mask_out, acc);
}

// one warp per output row
template <typename T>
__global__ void k_coarse_gemv(const double* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x,
                              const long long* __restrict__ gmap, long long n) {
  const long long warps = (long long)gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  for (long long i = blockIdx.x * (long long)(blockDim.x / 32) + (threadIdx.x >> 5); i < n; i += warps) {
    double acc = 0.0;
    const double* row = Ainv + i * n;
    for (long long j = lane; j < n; j += 32) acc = fma(row[j], (double)b[gmap[j]], acc);
    acc = warp_sum(acc);
    if (lane == 0) x[gmap[i]] = (T)acc;
  }
}

}  // namespace

cudaError_t dot_partial(const double* x, const double* y, long long n, double* partial, cudaStream_t s) {
  k_dot_partial<double><<<red_blocks(n), kThreads, 0, s>>>(x, y, n, partial);
  return counted(cudaGetLastError());
}
cudaError_t dot_partial_f32(const float* x, const float* y, long long n, double* partial, cudaStream_t s) {
  k_dot_partial<float><<<red_blocks(n), kThreads, 0, s>>>(x, y, n, partial);
  return counted(cudaGetLastError());
}

cudaError_t finish(const double* partial, long long n, double* S, int op, int idx, int aux, double* host_copy,
                   cudaStream_t s) {
  k_finish<<<1, kThreads, 0, s>>>(partial, red_blocks(n), S, op, idx, aux);
  cudaError_t e = counted(cudaGetLastError());
  if (e != cudaSuccess || host_copy == nullptr) return e;
  return cudaMemcpyAsync(host_copy, S + idx, sizeof(double), cudaMemcpyDeviceToHost, s);
}

cudaError_t pcg_update(double* u, double* r, const double* p, const double* h, long long n, const double* S,
                       double* partial, cudaStream_t s) {
  k_pcg_update<<<red_blocks(n), kThreads, 0, s>>>(u, r, p, h, n, S, partial);
  return counted(cudaGetLastError());
}

cudaError_t pcg_direction(double* p, const double* z, long long n, const double* S, cudaStream_t s) {
  k_pcg_dir<<<grid_for(n), kThreads, 0, s>>>(p, z, n, S);
  return counted(cudaGetLastError());
}

template <typename T>
cudaError_t jacobi_first(T* x, const T* b, const T* dinv, long long n, T omega, cudaStream_t s, T* r) {
  k_jacobi_first<T><<<grid_for(n), kThreads, 0, s>>>(x, b, dinv, n, omega, r);
  return counted(cudaGetLastError());
}
template <typename T>
cudaError_t jacobi_step(T* x, T* r, const T* b, const T* dinv, long long n, T omega, int reset, cudaStream_t s) {
  k_jacobi<T><<<grid_for(n), kThreads, 0, s>>>(x, r, b, dinv, n, omega, reset);
  return counted(cudaGetLastError());
}
template <typename T>
cudaError_t cheb_first(T* x, T* d, const T* b, const T* dinv, long long n, T inv_theta, cudaStream_t s, T* r) {
  k_cheb_first<T><<<grid_for(n), kThreads, 0, s>>>(x, d, b, dinv, n, inv_theta, r);
  return counted(cudaGetLastError());
}
template <typename T>
cudaError_t cheb_step(T* x, T* d, T* r, const T* b, const T* dinv, long long n, T c1, T c2, int reset,
                      cudaStream_t s) {
  k_cheb<T><<<grid_for(n), kThreads, 0, s>>>(x, d, r, b, dinv, n, c1, c2, reset);
  return counted(cudaGetLastError());
}
template cudaError_t jacobi_first<double>(double*, const double*, const double*, long long, double, cudaStream_t,
                                          double*);
template cudaError_t jacobi_first<float>(float*, const float*, const float*, long long, float, cudaStream_t, float*);
template cudaError_t jacobi_step<double>(double*, double*, const double*, const double*, long long, double, int,
                                         cudaStream_t);
template cudaError_t jacobi_step<float>(float*, float*, const float*, const float*, long long, float, int,
                                        cudaStream_t);
template cudaError_t cheb_first<double>(double*, double*, const double*, const double*, long long, double,
                                        cudaStream_t, double*);
template cudaError_t cheb_first<float>(float*, float*, const float*, const float*, long long, float, cudaStream_t,
                                       float*);
template cudaError_t cheb_step<double>(double*, double*, double*, const double*, const double*, long long, double,
                                       double, int, cudaStream_t);
template cudaError_t cheb_step<float>(float*, float*, float*, const float*, const float*, long long, float, float,
                                      int, cudaStream_t);

cudaError_t color_indicator(double* v, const Mesh& m, int period, int c0, int c1, int c2, cudaStream_t s) {
  k_color_indicator<<<grid_for(m.N), kThreads, 0, s>>>(v, m, period, c0, c1, c2);
  return counted(cudaGetLastError());
}

cudaError_t accum_abs(double* acc, const double* y, long long n, cudaStream_t s) {
  k_accum_abs<<<grid_for(n), kThreads, 0, s>>>(acc, y, n);
  return counted(cudaGetLastError());
}

cudaError_t dinv_from_diag(const double* diag, double* dinv, long long n, cudaStream_t s) {
  k_dinv<<<grid_for(n), kThreads, 0, s>>>(diag, dinv, n);
  return counted(cudaGetLastError());
}
cudaError_t mask_boundary(double* v, const Mesh& m, cudaStream_t s) {
  k_mask<<<grid_for(m.N), kThreads, 0, s>>>(v, m);
  return counted(cudaGetLastError());
}
cudaError_t copy_masked(double* dst, const double* src, const Mesh& m, cudaStream_t s) {
  k_copy_masked<<<grid_for(m.N), kThreads, 0, s>>>(dst, src, m);
  return counted(cudaGetLastError());
}
cudaError_t to_f32(float* dst, const double* src, long long n, cudaStream_t s) {
  k_to_f32<<<grid_for(n), kThreads, 0, s>>>(dst, src, n);
  return counted(cudaGetLastError());
}
cudaError_t to_f64(double* dst, const float* src, long long n, cudaStream_t s) {
  k_to_f64<<<grid_for(n), kThreads, 0, s>>>(dst, src, n);
  return counted(cudaGetLastError());
}
cudaError_t start_vector(double* v, const Mesh& m, unsigned long long seed, cudaStream_t s) {
  k_start<<<grid_for(m.N), kThreads, 0, s>>>(v, m, seed);
  return counted(cudaGetLastError());
}
cudaError_t project_out(double* w, const double* V, long long ldv, int cnt, long long n, double* partial,
                        double* c, double* H, int ldh, cudaStream_t s) {
  const int nb = red_blocks(n);
  k_multi_dot<<<dim3(nb, cnt), kThreads, 0, s>>>(V, ldv, w, n, partial);
  cudaError_t e = counted(cudaGetLastError());
  if (e != cudaSuccess) return e;
  k_multi_finish<<<cnt, kThreads, 0, s>>>(partial, nb, c, H, ldh);
  if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
  k_multi_axpy<<<grid_for(n), kThreads, 0, s>>>(w, V, ldv, cnt, c, n);
  return counted(cudaGetLastError());
}

cudaError_t scale_by(double* w, const double* dinv, long long n, cudaStream_t s) {
  k_scale_by<<<grid_for(n), kThreads, 0, s>>>(w, dinv, n);
  return counted(cudaGetLastError());
}
cudaError_t axpy_dev(double* y, const double* x, long long n, const double* coef, double sign, cudaStream_t s) {
  k_axpy_dev<<<grid_for(n), kThreads, 0, s>>>(y, x, n, coef, sign);
  return counted(cudaGetLastError());
}
cudaError_t div_dev(double* y, const double* x, long long n, const double* den, cudaStream_t s) {
  k_div_dev<<<grid_for(n), kThreads, 0, s>>>(y, x, n, den);
  return counted(cudaGetLastError());
}
cudaError_t copy_scalar(double* dst, const double* src, cudaStream_t s) {
  k_copy_scalar<<<1, 1, 0, s>>>(dst, src);
  return counted(cudaGetLastError());
}
cudaError_t bounded_wait_probe(unsigned polls, int* out_dev, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(polls, out_dev);
  return counted(cudaGetLastError());
}
cudaError_t set_solve_params(double* S, int* ctrl, double rtol, int maxit, int cap, cudaStream_t s) {
  k_set_params<<<1, 1, 0, s>>>(S, ctrl, rtol, maxit, cap);
  return counted(cudaGetLastError());
}
cudaError_t start_check(const double* S, int* ctrl, double* hist, cudaGraphConditionalHandle hw, cudaStream_t s) {
  k_start_check<<<1, 1, 0, s>>>(S, ctrl, hist, hw);
  return counted(cudaGetLastError());
}
cudaError_t step_check(const double* S, int* ctrl, double* hist, cudaGraphConditionalHandle hw,
                       cudaGraphConditionalHandle hi, int has_if, cudaStream_t s) {
  k_step_check<<<1, 1, 0, s>>>(S, ctrl, hist, hw, hi, has_if);
  return counted(cudaGetLastError());
}
cudaError_t axpy(double* y, const double* x, long long n, double a, cudaStream_t s) {
  k_axpy<<<grid_for(n), kThreads, 0, s>>>(y, x, n, a);
  return counted(cudaGetLastError());
}
cudaError_t node_coords(double* xyz, const Mesh& m, const double* gll, double amp, cudaStream_t s) {
  Gll g;
  for (int i = 0; i < kMaxN; ++i) g.r[i] = i <= m.p ? gll[i] : 0.0;
  k_node_coords<<<grid_for(m.N), kThreads, 0, s>>>(xyz, m, g, amp);
  return counted(cudaGetLastError());
}

template <typename T>
cudaError_t axis_pass(const T* in, T* out, const long long od[3], int axis, const Axis1D& M, int mask_in,
                      int mask_out, int accumulate, cudaStream_t s) {
  const long long tot = od[0] * od[1] * od[2];
  if (tot <= 0) return cudaSuccess;
  const long long tin = tot / od[axis] * M.n_in;
  if (tot >= (1LL << 31) || tin >= (1LL << 31)) return cudaErrorInvalidValue;  // 32-bit point indices
  const unsigned o0 = (unsigned)od[0], o1 = (unsigned)od[1], o2 = (unsigned)od[2];
  if (std::is_same<T, float>::value)
    k_axis<T, float><<<grid_for(tot), kThreads, 0, s>>>(in, out, o0, o1, o2, axis, M.n_in, M.rowptr,
                                                         M.col, M.val32, mask_in, mask_out, accumulate);
  else
    k_axis<T, double><<<grid_for(tot), kThreads, 0, s>>>(in, out, o0, o1, o2, axis, M.n_in, M.rowptr,
                                                          M.col, M.val, mask_in, mask_out, accumulate);
  return counted(cudaGetLastError());
}
template cudaError_t axis_pass<double>(const double*, double*, const long long*, int, const Axis1D&, int, int,
                                       int, cudaStream_t);
template cudaError_t axis_pass<float>(const float*, float*, const long long*, int, const Axis1D&, int, int, int,
                                      cudaStream_t);

namespace {
// C (ldc) = beta C + alpha A B for an M x N block of C, A: M x K (lda), B: K x N (ldb), K <= 32:
// one 64 x 64 tile of C per thread block, the tile's A rows and B columns staged in shared
// memory (zero outside the matrices), 4 x 4 outputs per thread; every global access is
// bounds-checked against M, N and K.
constexpr int kGemmK = 32;
__global__ void __launch_bounds__(256)
k_dgemm_k32(const int M, const int N, const int K, const double alpha, const double* __restrict__ A,
            const long long lda, const double* __restrict__ B, const long long ldb, const double beta,
            double* __restrict__ C, const long long ldc) {
  __shared__ double As[64][kGemmK + 1];
  __shared__ double Bs[kGemmK][64];
  const long long i0 = (long long)blockIdx.y * 64, j0 = (long long)blockIdx.x * 64;
  for (int idx = threadIdx.x; idx < 64 * K; idx += blockDim.x) {
    const int r = idx / K, k = idx - r * K;
    As[r][k] = (i0 + r < M) ? A[(i0 + r) * lda + k] : 0.0;
  }
  for (int idx = threadIdx.x; idx < K * 64; idx += blockDim.x) {
    const int k = idx >> 6, col = idx & 63;
    Bs[k][col] = (j0 + col < N) ? B[k * ldb + j0 + col] : 0.0;
  }
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  double acc[4][4] = {};
  for (int k = 0; k < K; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a[q] = As[ty + 16 * q][k];
      b[q] = Bs[k][tx + 16 * q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[q][w] = fma(a[q], b[w], acc[q][w]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const long long i = i0 + ty + 16 * q, j = j0 + tx + 16 * w;
      if (i < M && j < N) {
        double* o = C + i * ldc + j;
        *o = (beta == 0.0 ? 0.0 : beta * *o) + alpha * acc[q][w];
      }
    }
}

cudaError_t dgemm_k32(int M, int N, int K, double alpha, const double* A, long long lda, const double* B,
                      long long ldb, double beta, double* C, long long ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K < 1 || K > kGemmK) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
  k_dgemm_k32<<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  return counted(cudaGetLastError());
}
}  // namespace

size_t blocked_gj_work_doubles(long long n) { return (size_t)(2 * kGemmK * n + kGemmK * kGemmK); }

cudaError_t blocked_gauss_jordan_inverse(double* A, long long n, double* work, int* bad, cudaStream_t s) {
  constexpr int NB = kGemmK;
  double* R = work;                 // NB x n: the panel rows times the pivot block's inverse
  double* Cb = R + (size_t)NB * n;  // n x NB: the panel columns
  double* P = Cb + (size_t)n * NB;  // NB x NB: the pivot block, inverted in place
  const size_t w = sizeof(double);
  cudaError_t e = cudaSuccess;
  for (long long k0 = 0; k0 < n && e == cudaSuccess; k0 += NB) {
    const int b = (int)std::min<long long>(NB, n - k0);
    e = cudaMemcpy2DAsync(P, b * w, A + k0 * n + k0, n * w, b * w, b, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = launch_block_invert(P, 1, b, bad, s);
    if (e == cudaSuccess) e = dgemm_k32(b, (int)n, b, 1.0, P, b, A + k0 * n, n, 0.0, R, n, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Cb, b * w, A + k0, n * w, b * w, n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = dgemm_k32((int)n, (int)n, b, -1.0, Cb, b, R, n, 1.0, A, n, s);
    if (e == cudaSuccess) e = dgemm_k32((int)n, b, b, -1.0, Cb, b, P, b, 0.0, A + k0, n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(A + k0 * n, R, (size_t)b * n * w, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(A + k0 * n + k0, n * w, P, b * w, b * w, b, cudaMemcpyDeviceToDevice, s);
  }
  return e;
}

cudaError_t coarse_solve(const double* Ainv, const double* b, double* x, const long long* gmap, long long n,
                         cudaStream_t s) {
  long long g = (n + 7) / 8;
  if (g > (long long)device_sm_count() * 16) g = (long long)device_sm_count() * 16;
  k_coarse_gemv<double><<<(unsigned)g, kThreads, 0, s>>>(Ainv, b, x, gmap, n);
  return counted(cudaGetLastError());
}
cudaError_t coarse_solve_f32(const double* Ainv, const float* b, float* x, const long long* gmap, long long n,
                             cudaStream_t s) {
  long long g = (n + 7) / 8;
  if (g > (long long)device_sm_count() * 16) g = (long long)device_sm_count() * 16;
  k_coarse_gemv<float><<<(unsigned)g, kThreads, 0, s>>>(Ainv, b, x, gmap, n);
  return counted(cudaGetLastError());
}

}  // namespace hmg
