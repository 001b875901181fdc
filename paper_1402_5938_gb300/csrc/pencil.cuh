// Reduced-precision operator apply of the mixed V-cycle, "pencil" form: y += alpha * A x with
// FP32 vectors and arithmetic and geometric factors stored in FP32, FP16 (power-of-two scale per
// element) or BF16 (paper Sec. 2.3 matrix-free apply, sum factorization).
//
// This operator is bound by memory traffic (the factors: 24 or 12 bytes per Gauss point), so
// the kernel is shaped to issue as few instructions per flop as possible and to keep enough
// loads in flight, not for tensor cores: one thread owns one 1D line of an element in every
// direction (N^{d-1} threads per element, EPB elements per block, one tile per block), so every
// index is fixed per thread before the first phase and the unrolled contractions see compile-
// time offsets from a per-thread base, the 1D tables as uniform kernel-parameter operands and the
// line in registers. Passes are fused where a thread already holds the data:
//   3D: z-lines gather x and interpolate along z; y-lines interpolate along y; x-lines interpolate
//   along x and differentiate (u, u_x); y-lines differentiate (u_y) and z-lines differentiate (u_z,
//   kept in registers); z-lines then form v = G grad u at their points and apply D_z^T to v_z;
//   y-lines add D_y^T v_y; x-lines add D_x^T v_x and apply B_x^T; y-lines B_y^T; z-lines B_z^T and
//   scatter-add to y. Eight block barriers per tile.
//   2D: the same with x/y lines and four barriers.
// Tiles use a j-pitch of N rounded up to an odd number so that the x-line accesses of a warp hit
// distinct shared-memory banks. GPRE loads a thread's factors into registers before the first
// phase (small orders); otherwise they are read when needed, after a bulk L2 prefetch of the
// block's factor slab at the start.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "dispatch.cuh"

namespace hmg {

template <int DIM, int N>
struct PencilCfg {
  static constexpr int NL = DIM == 3 ? N * N : N;           // lines per direction per element
  static constexpr int NP = DIM == 3 ? N * N * N : N * N;   // points per element
  static constexpr int NC = DIM == 3 ? 6 : 3;
  static constexpr int PJ = (N % 2 == 0) ? N + 1 : N;       // j pitch (odd)
  static constexpr int PK = N * PJ;                          // k pitch (3D)
  static constexpr int EP = DIM == 3 ? N * PK : N * PJ;      // floats per element tile
  static constexpr int EPB0 = 128 / NL;
  static constexpr int EPB = (EPB0 >= 1 && EPB0 * NL >= 120) ? EPB0 : (256 / NL >= 1 ? 256 / NL : 1);
  static constexpr int LINES = EPB * NL;
  static constexpr int THREADS = (LINES + 31) / 32 * 32;
  static constexpr int NBUF = DIM == 3 ? 4 : 3;
  static constexpr size_t SMEM = (size_t)NBUF * EPB * EP * sizeof(float);
  // factors kept in registers from the start (GPRE) only while they stay few
  static constexpr bool PRE_OK = NC * N <= 42;
};

// The NC factors of point q of element e, as FP32. FP32: [e][NC][NP]; 16-bit: 3D point-major
// [e][NP][6] (three 32-bit words), 2D [e][3][NP]; FP16 values times the element's scale.
template <int DIM, int N, typename GT, typename T>
__device__ __forceinline__ void load_g(const GT* __restrict__ G, long long e, int q, float sc, T* g) {
  constexpr int NP = PencilCfg<DIM, N>::NP, NC = PencilCfg<DIM, N>::NC;
  if constexpr (std::is_same<GT, float>::value || std::is_same<GT, double>::value) {
    const GT* p = G + e * NC * NP + q;
#pragma unroll
    for (int c = 0; c < NC; ++c) g[c] = __ldg(p + c * NP);
  } else if constexpr (DIM == 3) {
    const unsigned* p = reinterpret_cast<const unsigned*>(G + (e * NP + q) * 6);
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      const unsigned v = __ldg(p + w);
      if constexpr (std::is_same<GT, __half>::value) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&v));
        g[2 * w] = f.x * sc;
        g[2 * w + 1] = f.y * sc;
      } else {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v));
        g[2 * w] = f.x;
        g[2 * w + 1] = f.y;
      }
    }
  } else {
    const GT* p = G + e * 3 * NP + q;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if constexpr (std::is_same<GT, __half>::value) g[c] = __half2float(p[c * NP]) * sc;
      else g[c] = __bfloat162float(p[c * NP]);
    }
  }
}

// out[i] = sum_m M[i*N + m] in[m] (TRN: M[m*N + i]), M a parameter-space table
template <int N, bool TRN, typename T>
__device__ __forceinline__ void mat1d(const T* __restrict__ M, const T* in, T* out) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T s = (TRN ? M[i] : M[i * N]) * in[0];
#pragma unroll
    for (int m = 1; m < N; ++m) s = fma(TRN ? M[m * N + i] : M[i * N + m], in[m], s);
    out[i] = s;
  }
}
// out[i] = acc[i] + sum_m M[m*N + i] in[m]
template <int N, typename T>
__device__ __forceinline__ void mat1d_t_acc(const T* __restrict__ M, const T* in, const T* acc, T* out) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T s = acc[i];
#pragma unroll
    for (int m = 0; m < N; ++m) s = fma(M[m * N + i], in[m], s);
    out[i] = s;
  }
}

// Byte range [lo, hi) rounded out to 16 bytes, prefetched into L2 by one bulk operation (the
// buffer holds >= 16 bytes of tail padding, so the rounded end stays inside the allocation).
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t lo = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~(uintptr_t)15;
  uintptr_t a = lo;
  while (a < hi) {  // one operation moves less than 2^20 bytes; slabs here are far smaller
    const uint32_t n = (uint32_t)((hi - a) < (1u << 19) ? (hi - a) : (1u << 19));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a), "r"(n) : "memory");
    a += n;
  }
}

// One tile: the EPB elements e0, e0 + 1, ... of mesh m (those below m.nelem), y += alpha A x, in
// value type T (float, or double for the batched FP64 operator) with factors of type GT; `smem`
// holds PencilCfg::SMEM bytes per value byte of float (scaled by sizeof(T) / 4).
template <int DIM, int N, typename T, typename GT, bool GPRE>
__device__ __forceinline__ void pencil_tile(const T* __restrict__ x, T* __restrict__ y, const GT* __restrict__ G,
                                            const float* __restrict__ gsc, const Mesh& m, const Tab<N, T>& tab,
                                            const T alpha, const long long e0, T* sm_pencil) {
  using C = PencilCfg<DIM, N>;
  constexpr int NL = C::NL, NP = C::NP, NC = C::NC, PJ = C::PJ, PK = C::PK, EP = C::EP, EPB = C::EPB;
  constexpr int TS = EPB * EP;       // values per buffer
  T* S = sm_pencil;                  // interpolation passes (forward and transposed)
  T* U = S + TS;                     // u at the Gauss points, later the transposed-derivative sum W
  T* GX = U + TS;                    // u_x, later v_x
  T* GY = GX + TS;                   // u_y, later v_y (3D)
  const int t = threadIdx.x;
  const int el = t / NL;
  const int l = t - el * NL;
  const long long e = e0 + el;
  // threads beyond the last line (the rest of the last warp) run every phase on element 0's tile
  // with their shared-memory stores switched off, so that all threads reach the same barriers
  const bool act = t < C::LINES;
  const bool valid = act && e < m.nelem;
  const int a = l % N, b = DIM == 3 ? l / N : 0;   // line coordinates
  const int eb = act ? el * EP : 0;
  if (t == 0) {
    const long long ne = (m.nelem - e0) < EPB ? (m.nelem - e0) : EPB;
    const size_t gbytes = sizeof(GT) * (size_t)NC * NP;
    bulk_prefetch_l2(reinterpret_cast<const char*>(G) + e0 * gbytes, ne * gbytes);
  }
  // element position, global node of the line's first node, and boundary masks
  long long nb = 0;
  int fl = 0;
  if (valid) {
    const int ex = (int)(e % m.E[0]);
    const long long r = e / m.E[0];
    const int ey = (int)(r % m.E[1]);
    const int ez = DIM == 3 ? (int)(r / m.E[1]) : 0;
    const long long base = ((long long)ez * m.p * m.Nn[1] + (long long)ey * m.p) * m.Nn[0] + (long long)ex * m.p;
    fl = (ex == 0) | ((ex == m.E[0] - 1) << 1) | ((ey == 0) << 2) | ((ey == m.E[1] - 1) << 3);
    if (DIM == 3) fl |= ((ez == 0) << 4) | ((ez == m.E[2] - 1) << 5);
    // 3D: this thread's z-line (i = a, j = b); 2D: its y-line (i = a)
    nb = base + a + (DIM == 3 ? (long long)b * m.Nn[0] : 0);
  }
  const long long sline = DIM == 3 ? m.Nn[0] * m.Nn[1] : m.Nn[0];  // node stride along the line
  // mask of the line's lateral position (i = a and, 3D, j = b) and of its two ends
  const bool bd_lat = ((a == 0) & (fl & 1)) | ((a == N - 1) & ((fl >> 1) & 1)) |
                      (DIM == 3 ? (((b == 0) & ((fl >> 2) & 1)) | ((b == N - 1) & ((fl >> 3) & 1))) : false);
  const int f_lo = DIM == 3 ? ((fl >> 4) & 1) : ((fl >> 2) & 1);
  const int f_hi = DIM == 3 ? ((fl >> 5) & 1) : ((fl >> 3) & 1);
  const float sc = (gsc != nullptr && valid) ? gsc[e] : 1.0f;

  // tile offsets: x-line (j = a, k = b) stride 1; y-line (i = a, k = b) stride PJ; z-line
  // (i = a, j = b) stride PK. 2D: x-line (j = a), y-line (i = a).
  const int ox = eb + a * PJ + (DIM == 3 ? b * PK : 0);
  const int oy = eb + a + (DIM == 3 ? b * PK : 0);
  const int oz = eb + a + b * PJ;

  T gpre[GPRE ? NC * N : 1];
  if constexpr (GPRE) {
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k)
        load_g<DIM, N, GT, T>(G, e, DIM == 3 ? a + b * N + k * N * N : a + k * N, sc, gpre + k * NC);
    }
  }
  T v[N], w[N];
  // ---- gather along the thread's line (z in 3D, y in 2D) and interpolate along it
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const bool bd = bd_lat | ((k == 0) & f_lo) | ((k == N - 1) & f_hi);
    v[k] = (valid && !bd) ? __ldg(x + nb + k * sline) : T(0);
  }
  mat1d<N, false>(tab.B, v, w);
  if (DIM == 3) {
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) S[oz + k * PK] = w[k];
    __syncthreads();
    // y-lines: interpolate along y
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = S[oy + k * PJ];
    mat1d<N, false>(tab.B, v, w);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) S[oy + k * PJ] = w[k];
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) S[oy + k * PJ] = w[k];
  }
  __syncthreads();
  // ---- x-lines: interpolate along x, differentiate along x
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = S[ox + k];
  mat1d<N, false>(tab.B, v, w);
  mat1d<N, false>(tab.D, w, v);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (act) U[ox + k] = w[k];
    if (act) GX[ox + k] = v[k];
  }
  __syncthreads();
  T uz[N];
  if (DIM == 3) {
    // y-lines: u_y; z-lines: u_z (kept in registers)
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = U[oy + k * PJ];
    mat1d<N, false>(tab.D, v, w);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) GY[oy + k * PJ] = w[k];
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = U[oz + k * PK];
    mat1d<N, false>(tab.D, v, uz);
    __syncthreads();
  } else {
    // 2D y-lines: u_y in registers
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = U[oy + k * PJ];
    mat1d<N, false>(tab.D, v, uz);
  }
  // ---- the thread's line (z in 3D, y in 2D): v = G grad u at its points, then D^T along it
  const int ol = DIM == 3 ? oz : oy;
  constexpr int SL = DIM == 3 ? PK : PJ;
  T vl[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T g[NC];
    if constexpr (GPRE) {
#pragma unroll
      for (int c = 0; c < NC; ++c) g[c] = gpre[k * NC + c];
    } else {
      if (valid) load_g<DIM, N, GT, T>(G, e, DIM == 3 ? a + b * N + k * N * N : a + k * N, sc, g);
      else {
#pragma unroll
        for (int c = 0; c < NC; ++c) g[c] = T(0);
      }
    }
    const T ux = GX[ol + k * SL];
    if (DIM == 3) {
      const T uy = GY[ol + k * SL];
      if (act) GX[ol + k * SL] = g[0] * ux + g[1] * uy + g[2] * uz[k];
      if (act) GY[ol + k * SL] = g[1] * ux + g[3] * uy + g[4] * uz[k];
      vl[k] = g[2] * ux + g[4] * uy + g[5] * uz[k];
    } else {
      if (act) GX[ol + k * SL] = g[0] * ux + g[1] * uz[k];
      vl[k] = g[1] * ux + g[2] * uz[k];
    }
  }
  mat1d<N, true>(tab.D, vl, w);
#pragma unroll
  for (int k = 0; k < N; ++k)
      if (act) U[ol + k * SL] = w[k];
  __syncthreads();
  if (DIM == 3) {
    // y-lines: W += D_y^T v_y
#pragma unroll
    for (int k = 0; k < N; ++k) {
      v[k] = GY[oy + k * PJ];
      vl[k] = U[oy + k * PJ];
    }
    mat1d_t_acc<N>(tab.D, v, vl, w);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) U[oy + k * PJ] = w[k];
    __syncthreads();
  }
  // ---- x-lines: W += D_x^T v_x, then B_x^T
#pragma unroll
  for (int k = 0; k < N; ++k) {
    v[k] = GX[ox + k];
    vl[k] = U[ox + k];
  }
  mat1d_t_acc<N>(tab.D, v, vl, w);
  mat1d<N, true>(tab.B, w, v);
#pragma unroll
  for (int k = 0; k < N; ++k)
      if (act) S[ox + k] = v[k];
  __syncthreads();
  if (DIM == 3) {
    // y-lines: B_y^T
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = S[oy + k * PJ];
    mat1d<N, true>(tab.B, v, w);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) S[oy + k * PJ] = w[k];
    __syncthreads();
  }
  // ---- the thread's line: B^T along it and scatter-add
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = S[ol + k * SL];
  mat1d<N, true>(tab.B, v, w);
  if (valid) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const bool bd = bd_lat | ((k == 0) & f_lo) | ((k == N - 1) & f_hi);
      if (!bd) atomicAdd(y + nb + k * sline, alpha * w[k]);
    }
  }
}

template <int DIM, int N, typename GT, bool GPRE>
__global__ void __launch_bounds__(PencilCfg<DIM, N>::THREADS)
k_apply_pencil(const float* __restrict__ x, float* __restrict__ y, const GT* __restrict__ G,
               const float* __restrict__ gsc, const Mesh m, const __grid_constant__ Tab<N, float> tab,
               const float alpha) {
  extern __shared__ __align__(16) float sm_pencil[];
  pencil_tile<DIM, N, float, GT, GPRE>(x, y, G, gsc, m, tab, alpha, (long long)blockIdx.x * PencilCfg<DIM, N>::EPB,
                                       sm_pencil);
}

// ---------------------------------------------------------------------------------------
// 3D "plane" form for small orders (N = p + 1 <= 5): a thread owns a whole 2D plane of an
// element and applies the two 1D tables of that plane's directions in registers, so only the
// changes of plane orientation go through shared memory (14 N^3 shared accesses per element
// against 23 N^3 for the line form, four barriers). Threads alternate between yz-planes
// (fixed x index: gather, z-interpolation, the pointwise factor product, the z and y transposed
// derivatives, the last transposed interpolation and the scatter, all along consecutive nodes in
// x across the lanes) and xy-planes (fixed z index: the x interpolation and derivative, the y
// derivative, the x transposed derivative and the x and y transposed interpolations):
//   yz(i):  x -> B_y, B_z                       -> S
//   xy(kq): S -> B_x = u, D_x u, D_y u          -> U, GX, S
//   yz(iq): U -> D_z u; G grad u; D_y^T v_y + D_z^T v_z -> U, v_x -> GX
//   xy(k):  U, GX -> + D_x^T v_x, B_x^T, B_y^T  -> S
//   yz(i):  S -> B_z^T, scatter-add
// Element tiles use the pitches j -> N, k -> PK with PK = 1 (mod 32) and an element stride of
// N PK = N (mod 32), so that the lanes of a warp, which run over (element, plane index),
// address 32 consecutive banks in both orientations.
// ---------------------------------------------------------------------------------------
constexpr bool plane_banks_ok(int N, int PK, int EPB, int threads) {
  const int EP = N * PK;
  for (int w = 0; w * 32 < threads; ++w) {
    for (int orient = 0; orient < 2; ++orient) {
      unsigned used = 0u;
      for (int lane = 0; lane < 32; ++lane) {
        const int t = 32 * w + lane;
        if (t >= EPB * N) continue;
        const int el = t / N, r = t % N;
        const int addr = el * EP + (orient == 0 ? r : r * PK);
        const unsigned bit = 1u << (addr % 32);
        if (used & bit) return false;
        used |= bit;
      }
    }
  }
  return true;
}
constexpr int plane_pk(int N, int EPB, int threads) {
  for (int pk = N * N; pk < N * N + 64; ++pk)
    if (plane_banks_ok(N, pk, EPB, threads)) return pk;
  return N * N;
}

template <int N>
struct PlaneCfg {
  static constexpr int NP = N * N * N, NC = 6;
  static constexpr int EPB = 128 / N;
  static constexpr int THREADS = (EPB * N + 31) / 32 * 32;
  static constexpr int PJ = N;
  static constexpr int PK = plane_pk(N, EPB, THREADS);
  static constexpr int EP = N * PK;
  static constexpr size_t SMEM = (size_t)3 * EPB * EP * sizeof(float);
};

template <int N, typename GT>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS, 4)
k_apply_plane(const float* __restrict__ x, float* __restrict__ y, const GT* __restrict__ G,
              const float* __restrict__ gsc, const Mesh m, const __grid_constant__ Tab<N, float> tab,
              const float alpha) {
  using C = PlaneCfg<N>;
  constexpr int NP = C::NP, NC = C::NC, PJ = C::PJ, PK = C::PK, EP = C::EP, EPB = C::EPB;
  extern __shared__ __align__(16) float sm_plane[];
  float* S = sm_plane;
  float* U = S + EPB * EP;
  float* GX = U + EPB * EP;
  const int t = threadIdx.x;
  const int el = t / N, r = t - (t / N) * N;   // element of the block, plane index
  const bool act = t < EPB * N;
  const long long e0 = (long long)blockIdx.x * EPB;
  const long long e = e0 + el;
  const bool valid = act && e < m.nelem;
  const int eb = act ? el * EP : 0;
  if (t == 0) {
    const long long ne = (m.nelem - e0) < EPB ? (m.nelem - e0) : EPB;
    const size_t gbytes = sizeof(GT) * (size_t)NC * NP;
    bulk_prefetch_l2(reinterpret_cast<const char*>(G) + e0 * gbytes, ne * gbytes);
  }
  long long base = 0;
  int fl = 0;
  if (valid) {
    const int ex = (int)(e % m.E[0]);
    const long long rr = e / m.E[0];
    const int ey = (int)(rr % m.E[1]);
    const int ez = (int)(rr / m.E[1]);
    base = ((long long)ez * m.p * m.Nn[1] + (long long)ey * m.p) * m.Nn[0] + (long long)ex * m.p;
    fl = (ex == 0) | ((ex == m.E[0] - 1) << 1) | ((ey == 0) << 2) | ((ey == m.E[1] - 1) << 3) |
         ((ez == 0) << 4) | ((ez == m.E[2] - 1) << 5);
  }
  const long long nx = m.Nn[0], nxy = m.Nn[0] * m.Nn[1];
  // yz-plane of this thread: x index i = r; its nodes' boundary mask
  const bool bd_x = ((r == 0) & (fl & 1)) | ((r == N - 1) & ((fl >> 1) & 1));
  auto bd_of = [&](int j, int k) -> bool {
    return bd_x | ((j == 0) & ((fl >> 2) & 1)) | ((j == N - 1) & ((fl >> 3) & 1)) | ((k == 0) & ((fl >> 4) & 1)) |
           ((k == N - 1) & ((fl >> 5) & 1));
  };
  const float sc = (gsc != nullptr && valid) ? gsc[e] : 1.0f;
  const int oyz = eb + r;             // yz-plane (i = r): + j * PJ + k * PK
  const int oxy = eb + r * PK;        // xy-plane (k = r): + i + j * PJ

  float A[N][N], Bv[N][N];
  // ---- yz(i): gather, B_y, B_z -> S
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < N; ++k)
      A[j][k] = (valid && !bd_of(j, k)) ? __ldg(x + base + r + j * nx + k * nxy) : 0.0f;
#pragma unroll
  for (int jq = 0; jq < N; ++jq)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      float s = tab.B[jq * N] * A[0][k];
#pragma unroll
      for (int j = 1; j < N; ++j) s = fmaf(tab.B[jq * N + j], A[j][k], s);
      Bv[jq][k] = s;
    }
#pragma unroll
  for (int jq = 0; jq < N; ++jq)
#pragma unroll
    for (int kq = 0; kq < N; ++kq) {
      float s = tab.B[kq * N] * Bv[jq][0];
#pragma unroll
      for (int k = 1; k < N; ++k) s = fmaf(tab.B[kq * N + k], Bv[jq][k], s);
      if (act) S[oyz + jq * PJ + kq * PK] = s;
    }
  __syncthreads();
  // ---- xy(kq): u = B_x, then D_x u -> GX, D_y u -> S (this plane's own region), u -> U
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int jq = 0; jq < N; ++jq) A[i][jq] = S[oxy + i + jq * PJ];
#pragma unroll
  for (int iq = 0; iq < N; ++iq)
#pragma unroll
    for (int jq = 0; jq < N; ++jq) {
      float s = tab.B[iq * N] * A[0][jq];
#pragma unroll
      for (int i = 1; i < N; ++i) s = fmaf(tab.B[iq * N + i], A[i][jq], s);
      Bv[iq][jq] = s;
      if (act) U[oxy + iq + jq * PJ] = s;
    }
#pragma unroll
  for (int iq = 0; iq < N; ++iq)
#pragma unroll
    for (int jq = 0; jq < N; ++jq) {
      float sx = tab.D[iq * N] * Bv[0][jq], sy = tab.D[jq * N] * Bv[iq][0];
#pragma unroll
      for (int m2 = 1; m2 < N; ++m2) {
        sx = fmaf(tab.D[iq * N + m2], Bv[m2][jq], sx);
        sy = fmaf(tab.D[jq * N + m2], Bv[iq][m2], sy);
      }
      if (act) GX[oxy + iq + jq * PJ] = sx;
      if (act) S[oxy + iq + jq * PJ] = sy;
    }
  __syncthreads();
  // ---- yz(iq): u_z = D_z u; v = G grad u; W = D_y^T v_y + D_z^T v_z -> U; v_x -> GX
#pragma unroll
  for (int jq = 0; jq < N; ++jq)
#pragma unroll
    for (int kq = 0; kq < N; ++kq) A[jq][kq] = U[oyz + jq * PJ + kq * PK];
  float VY[N][N];
#pragma unroll
  for (int jq = 0; jq < N; ++jq)
#pragma unroll
    for (int kq = 0; kq < N; ++kq) {
      float uz = tab.D[kq * N] * A[jq][0];
#pragma unroll
      for (int k2 = 1; k2 < N; ++k2) uz = fmaf(tab.D[kq * N + k2], A[jq][k2], uz);
      float g[NC];
      if (valid) load_g<3, N, GT, float>(G, e, r + N * jq + N * N * kq, sc, g);
      else {
#pragma unroll
        for (int c = 0; c < NC; ++c) g[c] = 0.0f;
      }
      const int o = oyz + jq * PJ + kq * PK;
      const float ux = GX[o], uy = S[o];
      if (act) GX[o] = g[0] * ux + g[1] * uy + g[2] * uz;
      VY[jq][kq] = g[1] * ux + g[3] * uy + g[4] * uz;
      Bv[jq][kq] = g[2] * ux + g[4] * uy + g[5] * uz;   // v_z
    }
#pragma unroll
  for (int jq = 0; jq < N; ++jq)
#pragma unroll
    for (int kq = 0; kq < N; ++kq) {
      float s = 0.0f;
#pragma unroll
      for (int m2 = 0; m2 < N; ++m2) {
        s = fmaf(tab.D[m2 * N + jq], VY[m2][kq], s);
        s = fmaf(tab.D[m2 * N + kq], Bv[jq][m2], s);
      }
      if (act) U[oyz + jq * PJ + kq * PK] = s;
    }
  __syncthreads();
  // ---- xy(k): W += D_x^T v_x; B_x^T; B_y^T -> S
#pragma unroll
  for (int iq = 0; iq < N; ++iq)
#pragma unroll
    for (int jq = 0; jq < N; ++jq) {
      A[iq][jq] = U[oxy + iq + jq * PJ];
      Bv[iq][jq] = GX[oxy + iq + jq * PJ];
    }
#pragma unroll
  for (int iq = 0; iq < N; ++iq)
#pragma unroll
    for (int jq = 0; jq < N; ++jq) {
      float s = A[iq][jq];
#pragma unroll
      for (int m2 = 0; m2 < N; ++m2) s = fmaf(tab.D[m2 * N + iq], Bv[m2][jq], s);
      VY[iq][jq] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int jq = 0; jq < N; ++jq) {
      float s = tab.B[i] * VY[0][jq];
#pragma unroll
      for (int iq = 1; iq < N; ++iq) s = fmaf(tab.B[iq * N + i], VY[iq][jq], s);
      A[i][jq] = s;
    }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float s = tab.B[j] * A[i][0];
#pragma unroll
      for (int jq = 1; jq < N; ++jq) s = fmaf(tab.B[jq * N + j], A[i][jq], s);
      if (act) S[oxy + i + j * PJ] = s;
    }
  __syncthreads();
  // ---- yz(i): B_z^T and scatter-add
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int kq = 0; kq < N; ++kq) A[j][kq] = S[oyz + j * PJ + kq * PK];
  if (valid) {
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float s = tab.B[k] * A[j][0];
#pragma unroll
        for (int kq = 1; kq < N; ++kq) s = fmaf(tab.B[kq * N + k], A[j][kq], s);
        if (!bd_of(j, k)) atomicAdd(y + base + r + j * nx + k * nxy, alpha * s);
      }
  }
}

// The plane form (3D, N <= kMaxNPlane) with factors of type GT.
constexpr int kMaxNPlane = 5;
template <int N, typename GT>
cudaError_t launch_plane(const Mesh& m, const Basis1D& b, const float* x, float* y, const GT* G, const float* gsc,
                         float alpha, cudaStream_t s) {
  using C = PlaneCfg<N>;
  const long long blocks = (m.nelem + C::EPB - 1) / C::EPB;
  if (blocks == 0) return cudaSuccess;
  auto kern = k_apply_plane<N, GT>;
  cudaError_t e = ensure_smem(kern, C::SMEM);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(x, y, G, gsc, m, make_tab<N, float>(b), alpha);
  return counted(cudaGetLastError());
}

// The pencil-form apply with factors of type GT: one tile of EPB elements per block.
template <int DIM, int N, typename GT>
cudaError_t launch_pencil(const Mesh& m, const Basis1D& b, const float* x, float* y, const GT* G, const float* gsc,
                          float alpha, bool pre, cudaStream_t s) {
  using C = PencilCfg<DIM, N>;
  const long long blocks = (m.nelem + C::EPB - 1) / C::EPB;
  if (blocks == 0) return cudaSuccess;
  if (pre && C::PRE_OK) {
    auto kern = k_apply_pencil<DIM, N, GT, C::PRE_OK>;
    cudaError_t e = ensure_smem(kern, C::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(x, y, G, gsc, m, make_tab<N, float>(b), alpha);
  } else {
    auto kern = k_apply_pencil<DIM, N, GT, false>;
    cudaError_t e = ensure_smem(kern, C::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(x, y, G, gsc, m, make_tab<N, float>(b), alpha);
  }
  return counted(cudaGetLastError());
}

}  // namespace hmg
