// Element kernels of the sum-factorized, matrix-free Q_p operator (templated on the
// dimension DIM, the 1D node count N = p+1 and the precision T).
//
// Every kernel stages `epb` consecutive elements per thread block in shared memory as
// tensor tiles t[k][j][i] (x fastest) and applies the 1D (N x N) tables along one
// direction at a time ("sum factorization": O(N^{d+1}) per element instead of O(N^{2d}),
// paper Sec. 2.3). A contraction phase gives each thread one whole 1D line: it reads the
// N line values into registers and applies the table with compile-time indices, so
// every table entry is a uniform (broadcast) operand read from the kernel's parameter
// space.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace hmg {

template <int DIM, int N>
struct Sh {
  static constexpr int NP = DIM == 3 ? N * N * N : N * N;  // points per element
  static constexpr int NL = DIM == 3 ? N * N : N;          // lines per direction
  static constexpr int NC = DIM == 3 ? 6 : 3;              // symmetric G components
};

// First element offset and node strides of line l along direction dir in a tile.
template <int DIM, int N>
__device__ __forceinline__ void line_of(int dir, int l, int& base, int& stride) {
  if (DIM == 2) {
    if (dir == 0) { base = l * N; stride = 1; }
    else { base = l; stride = N; }
  } else {
    const int a = l % N, b = l / N;
    if (dir == 0) { base = (b * N + a) * N; stride = 1; }
    else if (dir == 1) { base = b * N * N + a; stride = N; }
    else { base = b * N + a; stride = N * N; }
  }
}

// Global node number of local node `a` of element e; bd = node lies on the boundary.
template <int DIM, int N>
__device__ __forceinline__ long long elem_node(const Mesh& m, long long e, int a, bool& bd) {
  const int i = a % N;
  const int j = (a / N) % N;
  const long long ex = e % m.E[0];
  const long long r1 = e / m.E[0];
  const long long I = ex * m.p + i;
  long long J, K = 0;
  if (DIM == 3) {
    const int k = a / (N * N);
    const long long ey = r1 % m.E[1];
    const long long ez = r1 / m.E[1];
    J = ey * m.p + j;
    K = ez * m.p + k;
    bd = (I == 0) | (I == m.Nn[0] - 1) | (J == 0) | (J == m.Nn[1] - 1) | (K == 0) | (K == m.Nn[2] - 1);
    return (K * m.Nn[1] + J) * m.Nn[0] + I;
  } else {
    J = r1 * m.p + j;
    bd = (I == 0) | (I == m.Nn[0] - 1) | (J == 0) | (J == m.Nn[1] - 1);
    return J * m.Nn[0] + I;
  }
}

// Interior numbering (boundary nodes removed, x fastest) of an interior global node g.
template <int DIM>
__device__ __forceinline__ long long interior_index(const Mesh& m, long long g) {
  const long long I = g % m.Nn[0];
  const long long r = g / m.Nn[0];
  if (DIM == 3) {
    const long long J = r % m.Nn[1], K = r / m.Nn[1];
    return ((K - 1) * (m.Nn[1] - 2) + (J - 1)) * (m.Nn[0] - 2) + (I - 1);
  }
  return (r - 1) * (m.Nn[0] - 2) + (I - 1);
}

// Per-element gather/scatter data computed once per element tile: the global node number of
// local node (0,0,0) and six boundary-face bits (x0, x1, y0, y1, z0, z1).
__device__ __forceinline__ void elem_base(const Mesh& m, long long e, long long* base, int* flags) {
  const int ex = (int)(e % m.E[0]);
  const long long r = e / m.E[0];
  const int ey = (int)(r % m.E[1]);
  const int ez = (int)(r / m.E[1]);
  *base = ((long long)ez * m.p * m.Nn[1] + (long long)ey * m.p) * m.Nn[0] + (long long)ex * m.p;
  int f = (ex == 0) | ((ex == m.E[0] - 1) << 1) | ((ey == 0) << 2) | ((ey == m.E[1] - 1) << 3);
  if (m.dim == 3) f |= ((ez == 0) << 4) | ((ez == m.E[2] - 1) << 5);
  *flags = f;
}

// Global node of local point a of an element with the given base/flags (32-bit local math).
template <int DIM, int N>
__device__ __forceinline__ long long local_node(int a, long long base, int f, long long nx, long long nxy,
                                                bool& bd) {
  const int i = a % N, j = (a / N) % N, k = DIM == 3 ? a / (N * N) : 0;
  bd = ((i == 0) & (f & 1)) | ((i == N - 1) & ((f >> 1) & 1)) | ((j == 0) & ((f >> 2) & 1)) |
       ((j == N - 1) & ((f >> 3) & 1));
  if (DIM == 3) bd |= ((k == 0) & ((f >> 4) & 1)) | ((k == N - 1) & ((f >> 5) & 1));
  return base + (long long)k * nxy + (long long)j * nx + i;
}

// dst (=, or += if ACC) table contraction of src along `dir` for the `ne` tiles of the block.
//   TRN = false: out[i] = sum_m M[i*N+m] in[m]   (nodes -> Gauss points)
//   TRN = true : out[i] = sum_m M[m*N+i] in[m]   (transpose, Gauss points -> nodes)
// src may equal dst: each thread reads its whole line before writing it.
template <int DIM, int N, typename T, bool TRN, bool ACC>
__device__ __forceinline__ void contract(const T* src, T* dst, const T* M, int dir, int ne) {
  constexpr int NP = Sh<DIM, N>::NP, NL = Sh<DIM, N>::NL;
  const int total = ne * NL;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int e = t / NL, l = t - e * NL;
    int base, stride;
    line_of<DIM, N>(dir, l, base, stride);
    base += e * NP;
    T in[N];
#pragma unroll
    for (int m = 0; m < N; ++m) in[m] = src[base + m * stride];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s = (TRN ? M[i] : M[i * N]) * in[0];
#pragma unroll
      for (int m = 1; m < N; ++m) s = fma(TRN ? M[m * N + i] : M[i * N + m], in[m], s);
      if (ACC) dst[base + i * stride] += s;
      else dst[base + i * stride] = s;
    }
  }
}

// Error code a kernel writes to its error flag when a bounded wait on a TMA copy gives up, and
// the poll limit of those waits.
constexpr int kErrTmaTimeout = 1;
constexpr uint32_t kWaitPolls = 1u << 22;

// ---------------------------------------------------------------------------------------
// FP64 apply, y += alpha * A x. On GB300 a warp-wide DFMA occupies the SM's FP64 pipe
// for ~16 cycles while shared-memory loads and integer work issue elsewhere, so this
// variant optimizes for full warps and balanced SMs rather than for few loads: one
// small thread block per group of NEG elements (no block-wide coupling between groups),
// one thread per output point in every contraction (so NEG*N^d work items fill warps
// for any N), tables and tiles in shared memory, per-element base offsets so the
// gather/scatter use 32-bit local index arithmetic.
// Buffers (4 per element tile): cur/nxt ping-pong for the B and B^T passes, and the
// reference gradient (V0 in the free ping-pong buffer, V1, V2).
// ---------------------------------------------------------------------------------------
// Block shapes of the FP64 apply: variant V in {0,1,2} of (elements per block NEG, threads GT);
// V = 3 is V = 2's shape with the geometric factors staged in shared memory by TMA.
// Low orders vary the elements per block (one warp's worth, ~128 or ~512 points); high orders
// keep one element per block and vary the threads. Setup times the variants on each level
// and keeps the fastest (see tune_apply in hmg.cu).
constexpr int apply64_gt_rule(int w) { return w <= 512 ? 32 : (w <= 1000 ? 64 : (w <= 2200 ? 128 : (w <= 3400 ? 256 : 512))); }
constexpr int apply64_neg(int np, int v) {
  return v == 3 ? apply64_neg(np, 2)   // variant 3: the shape of variant 2 with G staged by TMA
                : (np >= 100 ? 1 : ((v == 0 ? 32 : (v == 1 ? 128 : 512)) / np > 1 ? (v == 0 ? 32 : (v == 1 ? 128 : 512)) / np : 1));
}
constexpr int apply64_gt(int np, int v) {
  return v == 3 ? apply64_gt(np, 2) : np < 100 ? apply64_gt_rule(apply64_neg(np, v) * np)
                  : (v == 0 ? apply64_gt_rule(np)
                            : (v == 1 ? (2 * apply64_gt_rule(np) > 512 ? 512 : 2 * apply64_gt_rule(np))
                                      : (apply64_gt_rule(np) >= 64 ? apply64_gt_rule(np) / 2 : 4 * apply64_gt_rule(np))));
}

template <int DIM, int N, int V>
struct Apply64Cfg {
  static constexpr int NP = Sh<DIM, N>::NP;
  static constexpr int NC = Sh<DIM, N>::NC;
  static constexpr int NEG = apply64_neg(NP, V);
  static constexpr int W = NEG * NP;
  static constexpr int GT = apply64_gt(NP, V);
  // shared-memory layout (16-byte aligned regions): [mbarrier, flag | 16 B] [B, D tables]
  // [4 tiles of W] [element bases, face bits] [G slab of NEG elements + 16 B alignment slack]
  static constexpr size_t base_bytes = ((16 + (size_t)(2 * N * N + (DIM + 1) * W) * 8 + NEG * 16) + 15) & ~(size_t)15;
  static constexpr size_t gslab = (((size_t)W * NC * 8 + 16) + 15) & ~(size_t)15;
  // Variant 3 stages G with a bulk TMA copy that overlaps the gather and interpolation phases.
  // The kernel is FP64-pipe bound, so staging trades occupancy for load latency; the autotuner
  // keeps it only where it measures faster.
  static constexpr bool STAGE = V == 3 && base_bytes + gslab <= 200 * 1024;
  static constexpr size_t smem = base_bytes + (STAGE ? gslab : 0);
};

// sum_m M(idx, m) src[base + m*stride]  (TRN: M[m*N + idx], else M[idx*N + m])
template <int N, bool TRN>
__device__ __forceinline__ double pt_dot(const double* __restrict__ M, const double* src, int idx, int base,
                                         int stride) {
  double s = (TRN ? M[idx] : M[idx * N]) * src[base];
#pragma unroll
  for (int m = 1; m < N; ++m) s = fma(TRN ? M[m * N + idx] : M[idx * N + m], src[base + m * stride], s);
  return s;
}
// acc + the same sum (one FMA chain: no separate add per direction)
template <int N, bool TRN>
__device__ __forceinline__ double pt_dot_acc(const double* __restrict__ M, const double* src, int idx, int base,
                                             int stride, double acc) {
#pragma unroll
  for (int m = 0; m < N; ++m) acc = fma(TRN ? M[m * N + idx] : M[idx * N + m], src[base + m * stride], acc);
  return acc;
}

// Scale of the scatter-add: y += alpha * A x with alpha = +1 and -1 (every solver call) taken as
// a plain or negated add, so that no FP64 multiply is issued per node.
enum : int { kAlphaOne = 0, kAlphaMinusOne = 1, kAlphaOther = 2 };
inline int alpha_mode(double alpha) {
  return alpha == 1.0 ? kAlphaOne : (alpha == -1.0 ? kAlphaMinusOne : kAlphaOther);
}

// The work of one thread block of the FP64 apply: elements e0g, ..., e0g + NEG - 1 (those below
// m.nelem); smem_raw is the block's dynamic shared memory (Apply64Cfg::smem bytes).
template <int DIM, int N, int V>
__device__ __forceinline__ void apply64_tile(const double* __restrict__ x, double* __restrict__ y,
                                             const double* __restrict__ G, const Mesh& m, const Tab<N, double>& tab,
                                             const double alpha, const int amode, int* __restrict__ err,
                                             const long long e0g, unsigned char* smem_raw) {
  using C = Apply64Cfg<DIM, N, V>;
  constexpr int NP = C::NP, NEG = C::NEG, W = C::W, NC = Sh<DIM, N>::NC;
  constexpr int S1 = N, S2 = N * N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  int* sflag = reinterpret_cast<int*>(smem_raw + 8);
  const int neg = (int)min((long long)NEG, m.nelem - e0g);
  int goff = 0;  // byte offset of the staged slab above its 16-byte boundary
  unsigned char* gstage = smem_raw + C::base_bytes;
  if (C::STAGE) {
    const char* p = reinterpret_cast<const char*>(G + e0g * NC * NP);
    goff = (int)(reinterpret_cast<uintptr_t>(p) & 15);
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_init_fence();
      const uint32_t bytes = (uint32_t)(((long long)neg * NC * NP * 8 + goff + 15) & ~15LL);
      bulk_g2s(gstage, p - goff, bytes, bar);
    }
  }
  double* sB = reinterpret_cast<double*>(smem_raw + 16);
  double* sD = sB + N * N;
  double* T0 = sD + N * N;
  double* T1 = T0 + W;
  double* V1 = T1 + W;
  double* V2 = V1 + W;  // 3D only
  long long* ebase = reinterpret_cast<long long*>(T0 + (DIM + 1) * W);
  int* eflag = reinterpret_cast<int*>(ebase + NEG);
  const long long e0 = e0g;
  const int ne = neg;
  const int nt = ne * NP;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    sB[t] = tab.B[t];
    sD[t] = tab.D[t];
  }
  for (int e = threadIdx.x; e < ne; e += blockDim.x) elem_base(m, e0 + e, &ebase[e], &eflag[e]);
  __syncthreads();
  const long long nx = m.Nn[0], nxy = m.Nn[0] * m.Nn[1];
  auto node = [&](int t, bool& bd) -> long long {
    const int e = t / NP, a = t - (t / NP) * NP;
    const int i = a % N, j = (a / N) % N, k = DIM == 3 ? a / (N * N) : 0;
    const int f = eflag[e];
    bd = ((i == 0) & (f & 1)) | ((i == N - 1) & ((f >> 1) & 1)) | ((j == 0) & ((f >> 2) & 1)) |
         ((j == N - 1) & ((f >> 3) & 1));
    if (DIM == 3) bd |= ((k == 0) & ((f >> 4) & 1)) | ((k == N - 1) & ((f >> 5) & 1));
    return ebase[e] + (long long)k * nxy + (long long)j * nx + i;
  };
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    bool bd;
    const long long g = node(t, bd);
    T0[t] = bd ? 0.0 : x[g];
  }
  __syncthreads();
  double* cur = T0;
  double* nxt = T1;
  // interpolation to the Gauss points, one direction at a time
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? S1 : S2);
    for (int t = threadIdx.x; t < nt; t += 2 * blockDim.x) {  // two independent chains per thread
      const int t2 = t + blockDim.x;
      const int a = t % NP, a2 = t2 % NP;
      const int idx = d == 0 ? a % N : (d == 1 ? (a / N) % N : a / (N * N));
      const int idx2 = d == 0 ? a2 % N : (d == 1 ? (a2 / N) % N : a2 / (N * N));
      const double v1 = pt_dot<N, false>(sB, cur, idx, t - idx * st, st);
      if (t2 < nt) nxt[t2] = pt_dot<N, false>(sB, cur, idx2, t2 - idx2 * st, st);
      nxt[t] = v1;
    }
    __syncthreads();
    double* tmp = cur; cur = nxt; nxt = tmp;
  }
  // collocated reference gradient and the pointwise geometric factor
  double* V0 = nxt;
  const double* Gb = G + e0 * NC * NP;
  if (C::STAGE) {  // the slab's bulk copy: thread 0 waits with a limit, then all observe the phase
    if (threadIdx.x == 0) *sflag = mbar_wait(bar, 0, kWaitPolls) ? 0 : 1;
    __syncthreads();
    if (*sflag) {
      if (threadIdx.x == 0) atomicExch(err, kErrTmaTimeout);
      return;
    }
    mbar_wait(bar, 0, kWaitPolls);
    Gb = reinterpret_cast<const double*>(gstage + goff);
  }
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const int a = t % NP;
    const int i = a % N, j = (a / N) % N;
    const double* g = Gb + t / NP * NC * NP + a;
    if (DIM == 3) {
      const int k = a / (N * N);
      const double g00 = g[0], g01 = g[NP], g02 = g[2 * NP], g11 = g[3 * NP], g12 = g[4 * NP], g22 = g[5 * NP];
      const double u0 = pt_dot<N, false>(sD, cur, i, t - i, 1);
      const double u1 = pt_dot<N, false>(sD, cur, j, t - j * S1, S1);
      const double u2 = pt_dot<N, false>(sD, cur, k, t - k * S2, S2);
      V0[t] = g00 * u0 + g01 * u1 + g02 * u2;
      V1[t] = g01 * u0 + g11 * u1 + g12 * u2;
      V2[t] = g02 * u0 + g12 * u1 + g22 * u2;
    } else {
      const double g00 = g[0], g01 = g[NP], g11 = g[2 * NP];
      const double u0 = pt_dot<N, false>(sD, cur, i, t - i, 1);
      const double u1 = pt_dot<N, false>(sD, cur, j, t - j * S1, S1);
      V0[t] = g00 * u0 + g01 * u1;
      V1[t] = g01 * u0 + g11 * u1;
    }
  }
  __syncthreads();
  // transposed derivative, summed over directions, into cur
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const int a = t % NP;
    const int i = a % N, j = (a / N) % N;
    double s = pt_dot_acc<N, true>(sD, V1, j, t - j * S1, S1, pt_dot<N, true>(sD, V0, i, t - i, 1));
    if (DIM == 3) {
      const int k = a / (N * N);
      s = pt_dot_acc<N, true>(sD, V2, k, t - k * S2, S2, s);
    }
    cur[t] = s;
  }
  __syncthreads();
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? S1 : S2);
    for (int t = threadIdx.x; t < nt; t += 2 * blockDim.x) {
      const int t2 = t + blockDim.x;
      const int a = t % NP, a2 = t2 % NP;
      const int idx = d == 0 ? a % N : (d == 1 ? (a / N) % N : a / (N * N));
      const int idx2 = d == 0 ? a2 % N : (d == 1 ? (a2 / N) % N : a2 / (N * N));
      const double v1 = pt_dot<N, true>(sB, cur, idx, t - idx * st, st);
      if (t2 < nt) nxt[t2] = pt_dot<N, true>(sB, cur, idx2, t2 - idx2 * st, st);
      nxt[t] = v1;
    }
    __syncthreads();
    double* tmp = cur; cur = nxt; nxt = tmp;
  }
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    bool bd;
    const long long g = node(t, bd);
    if (!bd) {
      const double v = cur[t];
      atomicAdd(y + g, amode == kAlphaOne ? v : (amode == kAlphaMinusOne ? -v : alpha * v));
    }
  }
}

template <int DIM, int N, int V>
__global__ void __launch_bounds__(Apply64Cfg<DIM, N, V>::GT)
k_apply64(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ G, const Mesh m,
          const __grid_constant__ Tab<N, double> tab, const double alpha, const int amode, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  apply64_tile<DIM, N, V>(x, y, G, m, tab, alpha, amode, err, (long long)blockIdx.x * Apply64Cfg<DIM, N, V>::NEG,
                          smem_raw);
}

// ---------------------------------------------------------------------------------------
// FP64 apply with stored element matrices, y += alpha * A x: for low orders (N <= 3) the dense
// element matvec, 2 N^{2d} flops, is cheaper than the 24 N^4 + 15 N^3 of sum factorization (at
// N = 3: 1,458 against 2,349) for 8 N^{2d} bytes per element. A block holds EPB elements, one
// thread per element row: the element's x in shared memory (boundary nodes as 0), then
// y_a = sum_b K[b][a] x_b with K column-major so that a warp reads consecutive rows of one
// column, then a scatter-add to interior nodes.
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256)
k_apply_dense64(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ Ke,
                const Mesh m, const double alpha) {
  constexpr int NP = Sh<DIM, N>::NP;
  constexpr int EPB = 256 / NP;
  __shared__ double xs[EPB * NP];
  __shared__ long long ebase[EPB];
  __shared__ int eflag[EPB];
  const long long nx = m.Nn[0], nxy = m.Nn[0] * m.Nn[1];
  const long long ngroups = (m.nelem + EPB - 1) / EPB;
  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long long e0 = grp * EPB;
    const int ne = (int)min((long long)EPB, m.nelem - e0);
    if (threadIdx.x < ne) elem_base(m, e0 + threadIdx.x, &ebase[threadIdx.x], &eflag[threadIdx.x]);
    __syncthreads();
    const int e = threadIdx.x / NP, a = threadIdx.x - e * NP;
    bool bd = true;
    long long gn = 0;
    if (e < ne) {
      gn = local_node<DIM, N>(a, ebase[e], eflag[e], nx, nxy, bd);
      xs[threadIdx.x] = bd ? 0.0 : x[gn];
    }
    __syncthreads();
    if (e < ne && !bd) {
      const double* k = Ke + (e0 + e) * NP * NP + a;
      const double* xe = xs + e * NP;
      double acc = 0.0;
#pragma unroll
      for (int b = 0; b < NP; ++b) acc = fma(k[b * NP], xe[b], acc);
      atomicAdd(y + gn, alpha * acc);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Geometry, stage 1: node coordinates of every element node -- x = X + amp prod sin(pi X), or
// the given coords[c][global node] -- interpolated to the Gauss points (x_q) and
// differentiated (dx_c/dxi_d), written to J[e][c*(DIM+1) + s][NP] with s = 0 for x_q and
// s = 1+d for dx_c/dxi_d (isoparametric geometry, Sec. 2.3).
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256)
k_geom_stage(double* __restrict__ J, const Mesh m, const double warp_amp, const double* __restrict__ coords,
             const __grid_constant__ GeoTab<N> tab, const int epb) {
  constexpr int NP = Sh<DIM, N>::NP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* U = reinterpret_cast<double*>(smem_raw);
  double* V = U + epb * NP;
  const long long e0 = (long long)blockIdx.x * epb;
  const int ne = (int)min((long long)epb, m.nelem - e0);
  for (int c = 0; c < DIM; ++c) {
    for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
      const int e = t / NP, a = t - e * NP;
      const long long eg = e0 + e;
      if (coords != nullptr) {
        bool bd;
        U[t] = coords[c * m.N + elem_node<DIM, N>(m, eg, a, bd)];
        continue;
      }
      const int idx[3] = {a % N, (a / N) % N, a / (N * N)};
      const long long ee[3] = {eg % m.E[0], (eg / m.E[0]) % m.E[1], eg / ((long long)m.E[0] * m.E[1])};
      double X[3], s = 1.0;
      for (int d = 0; d < DIM; ++d) {
        X[d] = ((double)ee[d] + tab.r[idx[d]]) / (double)m.E[d];
        s *= sinpi(X[d]);
      }
      U[t] = X[c] + warp_amp * s;
    }
    __syncthreads();
    for (int d = 0; d < DIM; ++d) {
      contract<DIM, N, double, false, false>(U, U, tab.B, d, ne);
      __syncthreads();
    }
    for (int d = 0; d < DIM; ++d) contract<DIM, N, double, false, false>(U, V + d * epb * NP, tab.D, d, ne);
    __syncthreads();
    for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
      const int e = t / NP, q = t - e * NP;
      double* o = J + ((e0 + e) * (DIM * (DIM + 1)) + c * (DIM + 1)) * NP + q;
      o[0] = U[t];
      for (int d = 0; d < DIM; ++d) o[(1 + d) * NP] = V[d * epb * NP + t];
    }
    __syncthreads();
  }
}

// Geometry, stage 2: G = mu(x_q) w_q det(J) J^-1 J^-T (symmetric, NC entries) and
// w_q det(J), one thread per Gauss point; mu from the formula a + b sum cos^2(k pi x), or the
// given values mu_arr[e * NP + q]. Sets *bad where det J <= 0.
template <int DIM, int N>
__global__ void k_geom_point(const double* __restrict__ J, double* __restrict__ G,
                             double* __restrict__ wdetJ, const Mesh m, const double mu_a,
                             const double mu_b, const double mu_k, const double* __restrict__ mu_arr,
                             const __grid_constant__ GeoTab<N> tab, int* __restrict__ bad) {
  constexpr int NP = Sh<DIM, N>::NP, NC = Sh<DIM, N>::NC;
  const long long tot = m.nelem * NP;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / NP;
    const int q = (int)(t - e * NP);
    const double* src = J + e * (DIM * (DIM + 1)) * NP + q;
    double xq[3], A[3][3];
    for (int c = 0; c < DIM; ++c) {
      xq[c] = src[(c * (DIM + 1)) * NP];
      for (int d = 0; d < DIM; ++d) A[c][d] = src[(c * (DIM + 1) + 1 + d) * NP];
    }
    double mu = 0.0;
    if (mu_arr != nullptr) {
      mu = mu_arr[t];
    } else {
      for (int c = 0; c < DIM; ++c) {
        const double cs = cospi(mu_k * xq[c]);
        mu += cs * cs;
      }
      mu = mu_a + mu_b * mu;
    }
    double w = tab.w[q % N] * tab.w[(q / N) % N];
    if (DIM == 3) w *= tab.w[q / (N * N)];
    double* g = G + e * NC * NP + q;
    if (DIM == 3) {
      // adjugate: Jinv = adj / det, adj[i][c] = cofactor of A[c][i]
      double adj[3][3];
      adj[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
      adj[0][1] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
      adj[0][2] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
      adj[1][0] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
      adj[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
      adj[1][2] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
      adj[2][0] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
      adj[2][1] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
      adj[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
      const double det = A[0][0] * adj[0][0] + A[0][1] * adj[1][0] + A[0][2] * adj[2][0];
      if (!(det > 0.0)) atomicExch(bad, 1);
      const double s = mu * w / det;
      const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
      for (int c = 0; c < 6; ++c) {
        const int i = ii[c], j = jj[c];
        g[c * NP] = s * (adj[i][0] * adj[j][0] + adj[i][1] * adj[j][1] + adj[i][2] * adj[j][2]);
      }
      wdetJ[e * NP + q] = w * det;
    } else {
      const double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
      if (!(det > 0.0)) atomicExch(bad, 1);
      // adj = [[A11, -A01], [-A10, A00]]
      const double a00 = A[1][1], a01 = -A[0][1], a10 = -A[1][0], a11 = A[0][0];
      const double s = mu * w / det;
      g[0] = s * (a00 * a00 + a01 * a01);
      g[NP] = s * (a00 * a10 + a01 * a11);
      g[2 * NP] = s * (a10 * a10 + a11 * a11);
      wdetJ[e * NP + q] = w * det;
    }
  }
}

// Gauss-point coordinates out of the stage-1 buffer: xq[c][e * NP + q].
template <int DIM, int N>
__global__ void k_extract_xq(const double* __restrict__ J, double* __restrict__ xq, const Mesh m) {
  constexpr int NP = Sh<DIM, N>::NP;
  const long long tot = m.nelem * NP;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t / NP;
    const int q = (int)(t - e * NP);
    for (int c = 0; c < DIM; ++c) xq[c * tot + t] = J[(e * (DIM * (DIM + 1)) + c * (DIM + 1)) * NP + q];
  }
}

// GLL nodes on [0,1] of the finest level and of a coarser one (n0, nk <= kMaxN).
struct MapNodes {
  double r0[kMaxN];
  double rk[kMaxN];
};

// Node coordinates of a coarser level from the finest level's isoparametric map: each node's
// reference coordinate X (element ec of the coarse mesh, GLL node i) lies in the fine element
// ef = floor(X E0) along each axis (the last one at X = 1), at xi = X E0 - ef, where
// x(X) = sum over the fine element's nodes of x_a prod_axis l_{a_axis}(xi_axis) (Sec. 2.3's
// isoparametric geometry). Xk[c][node], X0[c][fine node].
template <int DIM>
__global__ void k_level_coords(const double* __restrict__ X0, const Mesh m0, const Mesh mk,
                               const __grid_constant__ MapNodes nodes, double* __restrict__ Xk) {
  const int n0 = m0.p + 1;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < mk.N;
       g += (long long)gridDim.x * blockDim.x) {
    long long I[3] = {g % mk.Nn[0], (g / mk.Nn[0]) % mk.Nn[1], DIM == 3 ? g / (mk.Nn[0] * mk.Nn[1]) : 0};
    long long ef[3] = {0, 0, 0};
    double w[3][kMaxN];
    for (int a = 0; a < DIM; ++a) {
      const long long ec = min(I[a] / mk.p, (long long)mk.E[a] - 1);
      const double X = ((double)ec + nodes.rk[I[a] - ec * mk.p]) / (double)mk.E[a];
      const double tt = X * (double)m0.E[a];
      long long f = (long long)floor(tt);
      f = max(0LL, min(f, (long long)m0.E[a] - 1));
      ef[a] = f;
      const double xi = tt - (double)f;
      for (int j = 0; j < n0; ++j) {
        double l = 1.0;
        for (int q = 0; q < n0; ++q)
          if (q != j) l *= (xi - nodes.r0[q]) / (nodes.r0[j] - nodes.r0[q]);
        w[a][j] = l;
      }
    }
    double x[3] = {0.0, 0.0, 0.0};
    const int nk2 = DIM == 3 ? n0 : 1;
    for (int k = 0; k < nk2; ++k)
      for (int j = 0; j < n0; ++j)
        for (int i = 0; i < n0; ++i) {
          const double wt = w[0][i] * w[1][j] * (DIM == 3 ? w[2][k] : 1.0);
          const long long node = ((DIM == 3 ? (ef[2] * m0.p + k) : 0) * m0.Nn[1] + ef[1] * m0.p + j) * m0.Nn[0] +
                                 ef[0] * m0.p + i;
          for (int c = 0; c < DIM; ++c) x[c] += wt * X0[c * m0.N + node];
        }
    for (int c = 0; c < DIM; ++c) Xk[c * mk.N + g] = x[c];
  }
}

// ---------------------------------------------------------------------------------------
// diag(A): diag_a = sum_q sum_ij G_ij (dphi_a/dxi_i)(dphi_a/dxi_j), sum-factorized per
// symmetric pair (i,j) with the 1D product tables BB, BD, DD; scatter-added (boundary skipped).
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256)
k_diag(const double* __restrict__ G, double* __restrict__ diag, const Mesh m,
       const __grid_constant__ GeoTab<N> tab, const int epb) {
  constexpr int NP = Sh<DIM, N>::NP, NC = Sh<DIM, N>::NC;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* U = reinterpret_cast<double*>(smem_raw);
  double* Dt = U + epb * NP;
  const long long e0 = (long long)blockIdx.x * epb;
  const int ne = (int)min((long long)epb, m.nelem - e0);
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) Dt[t] = 0.0;
  const int pi_[6] = {0, 0, 0, 1, 1, 2}, pj_[6] = {0, 1, 2, 1, 2, 2};
  const int qi_[3] = {0, 0, 1}, qj_[3] = {0, 1, 1};
  for (int c = 0; c < NC; ++c) {
    const int i = DIM == 3 ? pi_[c] : qi_[c];
    const int j = DIM == 3 ? pj_[c] : qj_[c];
    const double f = (i == j) ? 1.0 : 2.0;
    __syncthreads();
    for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
      const int e = t / NP, q = t - e * NP;
      U[t] = f * G[((e0 + e) * NC + c) * NP + q];
    }
    __syncthreads();
    for (int d = 0; d < DIM; ++d) {
      const int k = (d == i) + (d == j);
      if (k == 0) contract<DIM, N, double, true, false>(U, U, tab.BB, d, ne);
      else if (k == 1) contract<DIM, N, double, true, false>(U, U, tab.BD, d, ne);
      else contract<DIM, N, double, true, false>(U, U, tab.DD, d, ne);
      __syncthreads();
    }
    for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) Dt[t] += U[t];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
    const int e = t / NP, a = t - e * NP;
    bool bd;
    const long long g = elem_node<DIM, N>(m, e0 + e, a, bd);
    if (!bd) atomicAdd(diag + g, Dt[t]);
  }
}

// ---------------------------------------------------------------------------------------
// b += M f (load vector of the nodal interpolant, Sec. 2.1 f_k): B to Gauss points, times
// w det J, B^T back, scatter-add to interior nodes. f is read at all nodes.
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
__global__ void __launch_bounds__(256)
k_mass(const double* __restrict__ f, double* __restrict__ b, const double* __restrict__ wdetJ,
       const Mesh m, const __grid_constant__ GeoTab<N> tab, const int epb) {
  constexpr int NP = Sh<DIM, N>::NP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* U = reinterpret_cast<double*>(smem_raw);
  const long long e0 = (long long)blockIdx.x * epb;
  const int ne = (int)min((long long)epb, m.nelem - e0);
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
    const int e = t / NP, a = t - e * NP;
    bool bd;
    U[t] = f[elem_node<DIM, N>(m, e0 + e, a, bd)];
  }
  __syncthreads();
  for (int d = 0; d < DIM; ++d) {
    contract<DIM, N, double, false, false>(U, U, tab.B, d, ne);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) U[t] *= wdetJ[e0 * NP + t];
  __syncthreads();
  for (int d = 0; d < DIM; ++d) {
    contract<DIM, N, double, true, false>(U, U, tab.B, d, ne);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
    const int e = t / NP, a = t - e * NP;
    bool bd;
    const long long g = elem_node<DIM, N>(m, e0 + e, a, bd);
    if (!bd) atomicAdd(b + g, U[t]);
  }
}

// ---------------------------------------------------------------------------------------
// Dense interior operator of a (small, coarsest) level: every tile of a block is one
// (element e, local column b) pair; the element operator is applied to the unit vector
// e_b by the same sum-factorized phases as k_apply (column b of K_e), and K_e[a][b] is
// added into A[ia*nI + ib] for interior a and b (interior numbering, x fastest); or, with
// Ke != nullptr, stored as the element matrix Ke[(e * NP + b) * NP + a] (column-major); or,
// with Kb != nullptr, only the columns and rows of the element-interior local nodes (all
// local indices in 1..N-2, MI = (N-2)^DIM of them, x fastest) are formed and stored as the
// element's interior block Kb[(e * MI + c) * MI + r]. An element-interior node belongs to
// no other element, so this block of K_e is also the block of the assembled operator.
// ---------------------------------------------------------------------------------------
template <int DIM, int N>
__device__ __forceinline__ int interior_local(int c) {  // c-th element-interior local node
  constexpr int M = N > 2 ? N - 2 : 1;  // (N = 2 has no interior nodes and never gets here)
  const int i = c % M + 1, j = (c / M) % M + 1;
  return DIM == 3 ? (c / (M * M) + 1) * N * N + j * N + i : j * N + i;
}

template <int DIM, int N>
__global__ void __launch_bounds__(256)
k_elem_dense(const double* __restrict__ G, double* __restrict__ A, const Mesh m,
             const __grid_constant__ Tab<N, double> tab, const long long nI, const int epb,
             double* __restrict__ Ke, double* __restrict__ Kb) {
  constexpr int NP = Sh<DIM, N>::NP, NC = Sh<DIM, N>::NC;
  constexpr int MI = DIM == 3 ? (N - 2) * (N - 2) * (N - 2) : (N - 2) * (N - 2);
  const int ncol = Kb != nullptr ? MI : NP;  // columns (tiles) per element
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* U = reinterpret_cast<double*>(smem_raw);
  double* V = U + epb * NP;
  const long long t0 = (long long)blockIdx.x * epb;
  const long long ntiles = m.nelem * ncol;
  const int ne = (int)min((long long)epb, ntiles - t0);
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
    const int e = t / NP, a = t - e * NP;
    const int c = (int)((t0 + e) % ncol);
    const int b = Kb != nullptr ? interior_local<DIM, N>(c) : c;
    U[t] = (a == b) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int d = 0; d < DIM; ++d) {
    contract<DIM, N, double, false, false>(U, U, tab.B, d, ne);
    __syncthreads();
  }
  for (int d = 0; d < DIM; ++d) contract<DIM, N, double, false, false>(U, V + d * epb * NP, tab.D, d, ne);
  __syncthreads();
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
    const int e = t / NP, q = t - e * NP;
    const long long el = (t0 + e) / ncol;
    const double* g = G + el * NC * NP + q;
    if (DIM == 3) {
      const double u0 = V[t], u1 = V[epb * NP + t], u2 = V[2 * epb * NP + t];
      const double g00 = g[0], g01 = g[NP], g02 = g[2 * NP], g11 = g[3 * NP], g12 = g[4 * NP], g22 = g[5 * NP];
      V[t] = g00 * u0 + g01 * u1 + g02 * u2;
      V[epb * NP + t] = g01 * u0 + g11 * u1 + g12 * u2;
      V[2 * epb * NP + t] = g02 * u0 + g12 * u1 + g22 * u2;
    } else {
      const double u0 = V[t], u1 = V[epb * NP + t];
      const double g00 = g[0], g01 = g[NP], g11 = g[2 * NP];
      V[t] = g00 * u0 + g01 * u1;
      V[epb * NP + t] = g01 * u0 + g11 * u1;
    }
  }
  __syncthreads();
  contract<DIM, N, double, true, false>(V, U, tab.D, 0, ne);
  __syncthreads();
  contract<DIM, N, double, true, true>(V + epb * NP, U, tab.D, 1, ne);
  __syncthreads();
  if (DIM == 3) {
    contract<DIM, N, double, true, true>(V + 2 * epb * NP, U, tab.D, 2, ne);
    __syncthreads();
  }
  for (int d = 0; d < DIM; ++d) {
    contract<DIM, N, double, true, false>(U, U, tab.B, d, ne);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < ne * NP; t += blockDim.x) {
    const int e = t / NP, a = t - e * NP;
    const long long el = (t0 + e) / ncol;
    const int b = (int)((t0 + e) % ncol);
    if (Kb != nullptr) {  // interior rows of interior column b (here the column index c)
      constexpr int M = N - 2;
      const int i = a % N, j = (a / N) % N, k = DIM == 3 ? a / (N * N) : 1;
      if (i >= 1 && i <= M && j >= 1 && j <= M && k >= 1 && k <= M) {
        const int r = (i - 1) + M * (j - 1) + (DIM == 3 ? M * M * (k - 1) : 0);
        Kb[(el * MI + b) * MI + r] = U[t];
      }
      continue;
    }
    if (Ke != nullptr) {
      Ke[(el * NP + b) * NP + a] = U[t];
      continue;
    }
    bool bda, bdb;
    const long long ga = elem_node<DIM, N>(m, el, a, bda);
    const long long gb = elem_node<DIM, N>(m, el, b, bdb);
    if (!bda && !bdb) atomicAdd(A + interior_index<DIM>(m, ga) * nI + interior_index<DIM>(m, gb), U[t]);
  }
}

}  // namespace hmg
