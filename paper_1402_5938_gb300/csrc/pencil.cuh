// Reduced-precision operator apply of the mixed V-cycle, "pencil" form: y += alpha * A x with
// FP32 vectors and arithmetic, the geometric factors stored in FP32, FP16 or BF16 (the 16-bit
// formats divided by a power-of-two scale per element) (paper Sec. 2.3 matrix-free apply, sum
// factorization).
//
// This operator is bound by memory traffic (the factors: 24 or 12 bytes per Gauss point), so the
// kernel is shaped to issue few instructions per flop and to keep every memory path busy with
// whole transactions, not for tensor cores: one thread owns one 1D line of an element in every
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
// Lanes run over the block's elements first (element = thread mod EPB, line = thread / EPB), and
// the tile pitches (PJ, PK, element stride EP) are chosen per order so that the lanes of a warp
// address distinct shared-memory banks in all line orientations. The factors are stored grouped
// by block, element innermost ([group][component][point][element]), so that a warp's factor load
// is one contiguous run; consecutive elements of a group are consecutive in x, so the gather and
// the scatter of a warp also touch runs of consecutive nodes. A thread's factors are loaded into
// registers one phase before the pointwise product (after a bulk L2 prefetch of the block's factor
// slab at the start), before the first phase (small orders), or at their use: three variants
// that trade load latency against registers, chosen per level by timing; prefetched factors stay
// in their stored form (16-bit pairs) until the pointwise product converts them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "dispatch.cuh"

namespace hmg {

// Elements per block and tile pitches of the pencil form, per dimension and order: the smallest
// shared-memory tiles whose warp accesses are free of bank conflicts (or nearly so) with about
// 100-500 threads per block.
struct PencilShape {
  int epb, pj, pk, ep;
};
__host__ __device__ constexpr PencilShape pencil_shape(int dim, int n) {
  if (dim == 3) {
    switch (n) {
      case 2: return {32, 2, 4, 9};
      case 3: return {32, 3, 9, 27};
      case 4: return {8, 5, 20, 84};
      case 5: return {8, 5, 25, 132};
      case 6: return {8, 7, 42, 252};
      case 7: return {4, 7, 55, 392};
      case 8: return {4, 9, 72, 584};
      case 9: return {4, 9, 81, 744};
      case 10: return {4, 13, 130, 1304};
      case 11: return {4, 11, 123, 1368};
      case 12: return {2, 13, 156, 1872};
      case 13: return {3, 13, 173, 2251};
      case 14: return {2, 17, 238, 3344};
      case 15: return {2, 17, 255, 3856};
      case 16: return {2, 17, 272, 4368};
      default: return {1, 17, 289, 4913};
    }
  }
  switch (n) {
    case 2: return {64, 2, 0, 5};
    case 3: return {32, 3, 0, 9};
    case 4: return {32, 4, 0, 17};
    case 5: return {32, 5, 0, 25};
    case 6: return {16, 7, 0, 42};
    case 7: return {32, 7, 0, 49};
    case 8: return {16, 9, 0, 74};
    case 9: return {32, 9, 0, 81};
    case 10: return {16, 11, 0, 110};
    case 11: return {32, 11, 0, 121};
    case 12: return {8, 13, 0, 156};
    case 13: return {32, 13, 0, 169};
    case 14: return {16, 15, 0, 210};
    case 15: return {32, 15, 0, 225};
    case 16: return {8, 17, 0, 276};
    default: return {16, 17, 0, 290};
  }
}

template <int DIM, int N, typename T = float>
struct PencilCfg {
  static constexpr PencilShape SH = pencil_shape(DIM, N);
  static constexpr int NL = DIM == 3 ? N * N : N;           // lines per direction per element
  static constexpr int NP = DIM == 3 ? N * N * N : N * N;   // points per element
  static constexpr int NC = DIM == 3 ? 6 : 3;
  static constexpr int EPB = SH.epb, PJ = SH.pj, PK = SH.pk, EP = SH.ep;
  static_assert(PJ >= N && (DIM == 2 || (PK >= N * PJ && EP >= N * PK)) && (DIM == 3 || EP >= N * PJ),
                "tile pitches must not overlap");
  static constexpr int LINES = EPB * NL;
  static constexpr int THREADS = (LINES + 31) / 32 * 32;
  static constexpr int NBUF = DIM == 3 ? 4 : 3;
  static constexpr size_t SMEM = (size_t)NBUF * EPB * EP * sizeof(T);
};

// Values of the grouped factor layout of one level (elements padded to whole groups of EPB).
inline size_t pencil_factor_values(int dim, int n, long long nelem) {
  const PencilShape s = pencil_shape(dim, n);
  const long long groups = (nelem + s.epb - 1) / s.epb;
  const long long np = dim == 3 ? (long long)n * n * n : (long long)n * n;
  return (size_t)(groups * s.epb * (dim == 3 ? 6 : 3) * np);
}

// 1D tables of the pencil form: B (GLL -> Gauss interpolation, B[q][a]) and D (collocated Gauss
// derivative, D[q][s]) as plain N x N arrays, and the four products a line goes through (B, D,
// B^T, D^T) in even/odd form. B's nodes and points are symmetric about the element's centre, so
// A[N-1-i][N-1-j] = s A[i][j] with s = +1 for B and B^T, -1 for D and D^T; with e_j = x_j + x_{N-1-j},
// o_j = x_j - x_{N-1-j} (j < H = N/2) the product y = A x becomes, for i < H,
//   a_i = sum_j E_ij e_j (+ A_iH x_H for odd N),  b_i = sum_j O_ij o_j,  y_i = a_i + b_i,
//   y_{N-1-i} = s (a_i - b_i),
// E_ij = (A_ij + A_i,N-1-j) / 2, O_ij = (A_ij - A_i,N-1-j) / 2, and for odd N the middle output
// y_H = sum_j A_Hj (e_j or o_j) (+ A_HH x_H for s = +1): 21 operations instead of 25 at N = 5, 57
// instead of 81 at N = 9, 177 instead of 289 at N = 17. Packing of each even/odd table: E at
// [0, H^2), O at [H^2, 2H^2), the middle column A_iH at [2H^2, 2H^2 + H), the middle row A_Hj at
// [2H^2 + H, 2H^2 + 2H), A_HH at 2H^2 + 2H.
template <int N, typename T>
struct PencilTab {
  T B[N * N];
  T D[N * N];
  T eB[N * N], eD[N * N], eBt[N * N], eDt[N * N];
};
// Even/odd products pay from N = 5 on (N = 2..4 break even or lose).
template <int N>
constexpr bool kUseEvenOdd = N >= 5;

inline void pack_even_odd(int n, const double* A /* A[i * n + j] */, double* out) {
  const int h = n / 2;
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < h; ++j) {
      out[i * h + j] = 0.5 * (A[i * n + j] + A[i * n + n - 1 - j]);
      out[h * h + i * h + j] = 0.5 * (A[i * n + j] - A[i * n + n - 1 - j]);
    }
  if (n % 2) {
    for (int i = 0; i < h; ++i) out[2 * h * h + i] = A[i * n + h];
    for (int j = 0; j < h; ++j) out[2 * h * h + h + j] = A[h * n + j];
    out[2 * h * h + 2 * h] = A[h * n + h];
  }
}

template <int N, typename T>
PencilTab<N, T> make_pencil_tab(const Basis1D& b) {
  PencilTab<N, T> t{};
  double Bt[N * N], Dt[N * N], pk[N * N];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      t.B[i * N + j] = (T)b.B[i * N + j];
      t.D[i * N + j] = (T)b.D[i * N + j];
      Bt[i * N + j] = b.B[j * N + i];
      Dt[i * N + j] = b.D[j * N + i];
    }
  const double* src[4] = {b.B, b.D, Bt, Dt};
  T* dst[4] = {t.eB, t.eD, t.eBt, t.eDt};
  for (int k = 0; k < 4; ++k) {
    for (int i = 0; i < N * N; ++i) pk[i] = 0.0;
    pack_even_odd(N, src[k], pk);
    for (int i = 0; i < N * N; ++i) dst[k][i] = (T)pk[i];
  }
  return t;
}

// Words of point q's factors as stored, so that prefetched factors keep their stored width
// (16-bit: half the registers of FP32 values) until unpack_g converts them at their use.
// Grouped layouts (FP32, FP16, BF16): RW words per point, 32-bit words (FP32 values; 16-bit 3D
// three component pairs; 16-bit 2D three values, one per word). FP64 factors are read from the
// element-major layout G[e][c][q] of the FP64 operator, NC doubles per point; double-float factors
// (df64) from the same layout, NC float pairs per point.
template <int DIM, typename GT>
struct RawG {
  static constexpr bool EM = std::is_same<GT, double>::value || std::is_same<GT, df64>::value;  // element-major
  using W = typename std::conditional<EM, GT, uint32_t>::type;
  static constexpr int RW = EM ? (DIM == 3 ? 6 : 3) : std::is_same<GT, float>::value ? (DIM == 3 ? 6 : 3) : 3;
};
template <int DIM, int N, typename GT>
__device__ __forceinline__ void load_raw(const GT* __restrict__ G, long long g, int el, int q,
                                         typename RawG<DIM, GT>::W* w) {
  using C = PencilCfg<DIM, N>;
  constexpr int NP = C::NP, NC = C::NC, EPB = C::EPB;
  if constexpr (std::is_same<GT, double>::value) {
    const double* p = G + (g * EPB + el) * NC * NP + q;
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = __ldg(p + c * NP);
  } else if constexpr (std::is_same<GT, df64>::value) {
    const float2* p = reinterpret_cast<const float2*>(G) + (g * EPB + el) * NC * NP + q;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float2 f = __ldg(p + c * NP);
      w[c] = df64(f.x, f.y);
    }
  } else if constexpr (std::is_same<GT, float>::value) {
    const float* p = G + (g * NC * NP + q) * EPB + el;
#pragma unroll
    for (int c = 0; c < NC; ++c) w[c] = __float_as_uint(__ldg(p + (long long)c * NP * EPB));
  } else if constexpr (DIM == 3) {
    const unsigned* p = reinterpret_cast<const unsigned*>(G) + (g * 3 * NP + q) * EPB + el;
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = __ldg(p + (long long)c * NP * EPB);
  } else {
    const unsigned short* p = reinterpret_cast<const unsigned short*>(G) + (g * 3 * NP + q) * EPB + el;
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = __ldg(p + (long long)c * NP * EPB);
  }
}
template <int DIM, typename GT, typename T>
__device__ __forceinline__ void unpack_g(const typename RawG<DIM, GT>::W* w, T* v) {
  if constexpr (std::is_same<GT, double>::value || std::is_same<GT, df64>::value) {
#pragma unroll
    for (int c = 0; c < (DIM == 3 ? 6 : 3); ++c) v[c] = w[c];
  } else if constexpr (std::is_same<GT, float>::value) {
#pragma unroll
    for (int c = 0; c < (DIM == 3 ? 6 : 3); ++c) v[c] = __uint_as_float(w[c]);
  } else if constexpr (DIM == 3) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 f;
      if constexpr (std::is_same<GT, __half>::value) f = __half22float2(*reinterpret_cast<const __half2*>(&w[c]));
      else f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[c]));
      v[2 * c] = f.x;
      v[2 * c + 1] = f.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const unsigned short u = (unsigned short)w[c];
      if constexpr (std::is_same<GT, __half>::value) v[c] = __half2float(__ushort_as_half(u));
      else v[c] = __bfloat162float(__ushort_as_bfloat16(u));
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
    for (int m = 1; m < N; ++m) s = fmadd(TRN ? M[m * N + i] : M[i * N + m], in[m], s);
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
    for (int m = 0; m < N; ++m) s = fmadd(M[m * N + i], in[m], s);
    out[i] = s;
  }
}
// out = A in with A given by its even/odd packing Q (PencilTab) and symmetry sign S
template <int N, int S, typename T>
__device__ __forceinline__ void mat1d_eo(const T* __restrict__ Q, const T* in, T* out) {
  constexpr int H = N / 2;
  constexpr bool ODD = (N & 1) != 0;
  T e[H], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = in[j] + in[N - 1 - j];
    o[j] = in[j] - in[N - 1 - j];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T a = Q[i * H] * e[0];
#pragma unroll
    for (int j = 1; j < H; ++j) a = fmadd(Q[i * H + j], e[j], a);
    if constexpr (ODD) a = fmadd(Q[2 * H * H + i], in[H], a);
    T b = Q[H * H + i * H] * o[0];
#pragma unroll
    for (int j = 1; j < H; ++j) b = fmadd(Q[H * H + i * H + j], o[j], b);
    out[i] = a + b;
    out[N - 1 - i] = S > 0 ? a - b : b - a;
  }
  if constexpr (ODD) {
    if constexpr (S > 0) {
      T c = Q[2 * H * H + 2 * H] * in[H];
#pragma unroll
      for (int j = 0; j < H; ++j) c = fmadd(Q[2 * H * H + H + j], e[j], c);
      out[H] = c;
    } else {
      T c = Q[2 * H * H + H] * o[0];
#pragma unroll
      for (int j = 1; j < H; ++j) c = fmadd(Q[2 * H * H + H + j], o[j], c);
      out[H] = c;
    }
  }
}
// The four line products of the pencil form: even/odd where that saves operations, else plain.
template <int N, typename T>
__device__ __forceinline__ void line_B(const PencilTab<N, T>& t, const T* in, T* out) {
  if constexpr (kUseEvenOdd<N>) mat1d_eo<N, 1>(t.eB, in, out);
  else mat1d<N, false>(t.B, in, out);
}
template <int N, typename T>
__device__ __forceinline__ void line_D(const PencilTab<N, T>& t, const T* in, T* out) {
  if constexpr (kUseEvenOdd<N>) mat1d_eo<N, -1>(t.eD, in, out);
  else mat1d<N, false>(t.D, in, out);
}
template <int N, typename T>
__device__ __forceinline__ void line_Bt(const PencilTab<N, T>& t, const T* in, T* out) {
  if constexpr (kUseEvenOdd<N>) mat1d_eo<N, 1>(t.eBt, in, out);
  else mat1d<N, true>(t.B, in, out);
}
template <int N, typename T>
__device__ __forceinline__ void line_Dt(const PencilTab<N, T>& t, const T* in, T* out) {
  if constexpr (kUseEvenOdd<N>) mat1d_eo<N, -1>(t.eDt, in, out);
  else mat1d<N, true>(t.D, in, out);
}

// Byte range [p, p + bytes) rounded out to 16 bytes and prefetched into L2 by bulk operations
// (the buffer holds >= 16 bytes of tail padding, so the rounded end stays inside the allocation).
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t lo = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~(uintptr_t)15;
  for (uintptr_t a = lo; a < hi;) {
    const uint32_t n = (uint32_t)((hi - a) < (1u << 19) ? (hi - a) : (1u << 19));
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a), "r"(n) : "memory");
    a += n;
  }
}

// One tile: the group g of EPB elements e0 = g * EPB, ... of mesh m (those below m.nelem),
// y += alpha A x in arithmetic T (FP32 with FP32 / 16-bit grouped factors, FP64 with the FP64
// operator's element-major factors, double-float with their float-pair split) on vectors of type
// X (T, or FP64 vectors for double-float arithmetic); `sm` holds PencilCfg<DIM, N, T>::SMEM bytes.
template <int DIM, int N, typename GT, int GM, typename T = float, typename X = T>
__device__ __forceinline__ void pencil_tile(const X* __restrict__ x, X* __restrict__ y,
                                            const GT* __restrict__ G, const float* __restrict__ gsc, const Mesh& m,
                                            const PencilTab<N, T>& tab, const T alpha, const long long g, T* sm) {
  using C = PencilCfg<DIM, N, T>;
  constexpr int NL = C::NL, NP = C::NP, NC = C::NC, PJ = C::PJ, PK = C::PK, EP = C::EP, EPB = C::EPB;
  constexpr int TS = EPB * EP;       // values per buffer
  T* S = sm;                         // interpolation passes (forward and transposed)
  T* U = S + TS;                     // u at the Gauss points, later the transposed-derivative sum W
  T* GX = U + TS;                    // u_x, later v_x
  T* GY = GX + TS;                   // u_y, later v_y (3D)
  const int t = threadIdx.x;
  const int el = t % EPB;            // element slot of the group
  const int l = t / EPB;             // line of the element
  // threads beyond the last line (the rest of the last warp) run every phase on element 0's tile
  // with their shared-memory stores switched off, so that all threads reach the same barriers
  const bool act = l < NL;
  const long long e0 = g * EPB;
  const long long e = e0 + el;
  const bool valid = act && e < m.nelem;
  const int a = act ? l % N : 0, b = (DIM == 3 && act) ? l / N : 0;   // line coordinates
  const int eb = act ? el * EP : 0;
  if (t == 0) {
    // the group's factors (element-major FP64: only the elements of the mesh, the allocation ends
    // at the last one; grouped layouts are padded to whole groups)
    const long long ng = RawG<DIM, GT>::EM ? (m.nelem - e0 < EPB ? m.nelem - e0 : EPB) : EPB;
    const size_t gbytes = sizeof(GT) * (size_t)NC * NP * EPB;
    bulk_prefetch_l2(reinterpret_cast<const char*>(G) + g * gbytes, sizeof(GT) * (size_t)NC * NP * ng);
  }
  // element position, global node of the line's first node, and boundary masks
  long long nb = 0;
  int fl = 0;
  if (valid) {
    // 32-bit decode (a level's element count is below 2^31): 64-bit divisions by runtime values
    // cost several times the instructions
    const unsigned ue = (unsigned)e, E0 = (unsigned)m.E[0], E1 = (unsigned)m.E[1];
    const unsigned ur = ue / E0;
    const int ex = (int)(ue - ur * E0);
    const int ey = (int)(ur % E1);
    const int ez = DIM == 3 ? (int)(ur / E1) : 0;
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
  // 16-bit factors are stored divided by a per-element power of two; the element's result is
  // scaled back at the scatter (exact, so the same as scaling each factor)
  const T asc = alpha * T((gsc != nullptr && valid) ? gsc[e] : 1.0f);

  // tile offsets: x-line (j = a, k = b) stride 1; y-line (i = a, k = b) stride PJ; z-line
  // (i = a, j = b) stride PK. 2D: x-line (j = a), y-line (i = a).
  const int ox = eb + a * PJ + (DIM == 3 ? b * PK : 0);
  const int oy = eb + a + (DIM == 3 ? b * PK : 0);
  const int oz = eb + a + b * PJ;
  auto qidx = [&](int k) { return DIM == 3 ? a + b * N + k * N * N : a + k * N; };

  constexpr bool GPRE = GM == 1;       // factors loaded before the first phase
  constexpr bool GAHEAD = GM == 0;     // ... one phase before the pointwise product
  constexpr int RW = RawG<DIM, GT>::RW;
  using GW = typename RawG<DIM, GT>::W;
  GW gpre[GPRE ? RW * N : 1];
  if constexpr (GPRE) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (valid) load_raw<DIM, N, GT>(G, g, el, qidx(k), gpre + k * RW);
      else {
#pragma unroll
        for (int c = 0; c < RW; ++c) gpre[k * RW + c] = GW(0);
      }
    }
  }
  T v[N], w[N];
  // ---- gather along the thread's line (z in 3D, y in 2D) and interpolate along it
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const bool bd = bd_lat | ((k == 0) & f_lo) | ((k == N - 1) & f_hi);
    v[k] = (valid && !bd) ? T(__ldg(x + nb + k * sline)) : T(0);
  }
  line_B<N>(tab, v, w);
  if (DIM == 3) {
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) S[oz + k * PK] = w[k];
    __syncthreads();
    // y-lines: interpolate along y
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = S[oy + k * PJ];
    line_B<N>(tab, v, w);
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
  line_B<N>(tab, v, w);
  line_D<N>(tab, w, v);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (act) U[ox + k] = w[k];
    if (act) GX[ox + k] = v[k];
  }
  __syncthreads();
  // the thread's factors: loaded here (unless GPRE loaded them at the start), one phase before
  // the pointwise product needs them, so that their latency overlaps the derivative phase
  GW gl[GAHEAD ? RW * N : 1];
  if constexpr (GAHEAD) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (valid) load_raw<DIM, N, GT>(G, g, el, qidx(k), gl + k * RW);
      else {
#pragma unroll
        for (int c = 0; c < RW; ++c) gl[k * RW + c] = GW(0);
      }
    }
  }
  T uz[N];
  if (DIM == 3) {
    // y-lines: u_y; z-lines: u_z (kept in registers)
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = U[oy + k * PJ];
    line_D<N>(tab, v, w);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) GY[oy + k * PJ] = w[k];
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = U[oz + k * PK];
    line_D<N>(tab, v, uz);
    __syncthreads();
  } else {
    // 2D y-lines: u_y in registers
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = U[oy + k * PJ];
    line_D<N>(tab, v, uz);
  }
  // ---- the thread's line (z in 3D, y in 2D): v = G grad u at its points, then D^T along it
  const int ol = DIM == 3 ? oz : oy;
  constexpr int SL = DIM == 3 ? PK : PJ;
  T vl[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    GW gj[GM == 2 ? RW : 1];
    if constexpr (GM == 2) {    // factors read at their use
      if (valid) load_raw<DIM, N, GT>(G, g, el, qidx(k), gj);
      else {
#pragma unroll
        for (int c = 0; c < RW; ++c) gj[c] = GW(0);
      }
    }
    T gv[NC];
    unpack_g<DIM, GT>(GM == 2 ? gj : (GPRE ? gpre + k * RW : gl + k * RW), gv);
    const T ux = GX[ol + k * SL];
    if (DIM == 3) {
      const T uy = GY[ol + k * SL];
      if (act) GX[ol + k * SL] = gv[0] * ux + gv[1] * uy + gv[2] * uz[k];
      if (act) GY[ol + k * SL] = gv[1] * ux + gv[3] * uy + gv[4] * uz[k];
      vl[k] = gv[2] * ux + gv[4] * uy + gv[5] * uz[k];
    } else {
      if (act) GX[ol + k * SL] = gv[0] * ux + gv[1] * uz[k];
      vl[k] = gv[1] * ux + gv[2] * uz[k];
    }
  }
  line_Dt<N>(tab, vl, w);
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
  line_Bt<N>(tab, w, v);
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (act) S[ox + k] = v[k];
  __syncthreads();
  if (DIM == 3) {
    // y-lines: B_y^T
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = S[oy + k * PJ];
    line_Bt<N>(tab, v, w);
#pragma unroll
    for (int k = 0; k < N; ++k)
      if (act) S[oy + k * PJ] = w[k];
    __syncthreads();
  }
  // ---- the thread's line: B^T along it and scatter-add
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = S[ol + k * SL];
  line_Bt<N>(tab, v, w);
  if (valid) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const bool bd = bd_lat | ((k == 0) & f_lo) | ((k == N - 1) & f_hi);
      if (!bd) atomicAdd(y + nb + k * sline, X(asc * w[k]));
    }
  }
}

template <int DIM, int N, typename GT, int GM, typename T, typename X>
__global__ void __launch_bounds__(PencilCfg<DIM, N, T>::THREADS)
k_apply_pencil(const X* __restrict__ x, X* __restrict__ y, const GT* __restrict__ G, const float* __restrict__ gsc,
               const Mesh m, const __grid_constant__ PencilTab<N, T> tab, const T alpha) {
  extern __shared__ __align__(16) unsigned char sm_pencil_raw[];
  pencil_tile<DIM, N, GT, GM, T, X>(x, y, G, gsc, m, tab, alpha, (long long)blockIdx.x,
                                    reinterpret_cast<T*>(sm_pencil_raw));
}

// The pencil-form apply: FP32 arithmetic with factors GT in the grouped layout, or FP64 arithmetic
// with the FP64 operator's factors (GT = T = double); one group per block.
// variant (GM): 0 factors loaded one phase before the pointwise product, 1 before the first phase
// (orders with few factors per line; else as 0), 2 at their use.
template <int DIM, int N, typename GT, int GM, typename T, typename X = T>
cudaError_t launch_pencil_gm(const Mesh& m, const Basis1D& b, const X* x, X* y, const GT* G, const float* gsc,
                             T alpha, cudaStream_t s) {
  using C = PencilCfg<DIM, N, T>;
  const long long blocks = (m.nelem + C::EPB - 1) / C::EPB;
  if (blocks == 0) return cudaSuccess;
  auto kern = k_apply_pencil<DIM, N, GT, GM, T, X>;
  cudaError_t e = ensure_smem(kern, C::SMEM);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(x, y, G, gsc, m, make_pencil_tab<N, T>(b), alpha);
  return counted(cudaGetLastError());
}
template <int DIM, int N, typename GT, typename T = float>
cudaError_t launch_pencil(const Mesh& m, const Basis1D& b, const T* x, T* y, const GT* G, const float* gsc,
                          T alpha, int variant, cudaStream_t s) {
  if (variant == 2) return launch_pencil_gm<DIM, N, GT, 2, T>(m, b, x, y, G, gsc, alpha, s);
  // factors kept in registers from the start only while they stay few
  if (variant == 1 && RawG<DIM, GT>::RW * N <= 42) return launch_pencil_gm<DIM, N, GT, 1, T>(m, b, x, y, G, gsc, alpha, s);
  return launch_pencil_gm<DIM, N, GT, 0, T>(m, b, x, y, G, gsc, alpha, s);
}

// Grouped reduced-precision factors of one element per block from G[e][c][q] (FP64): FP32 as
// they are (gsc = nullptr); FP16 and BF16 divided by gsc[e], the power of two that puts the
// element's largest |G| / gsc in [0.5, 1). Layouts as load_raw reads them; the buffer is zero-filled
// beforehand, so the padding elements of the last group stay zero.
template <typename GT>
__global__ void k_pack_grouped(const double* __restrict__ G, GT* __restrict__ out, float* __restrict__ gsc,
                               long long nelem, int dim, int np, int epb) {
  const long long e = blockIdx.x;
  if (e >= nelem) return;
  const int nc = dim == 3 ? 6 : 3;
  const int per_elem = nc * np;
  const double* ge = G + e * per_elem;
  double sc = 1.0;
  if (gsc != nullptr) {
    __shared__ double red[32];
    double amax = 0.0;
    for (int i = threadIdx.x; i < per_elem; i += blockDim.x) amax = fmax(amax, fabs(ge[i]));
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    int ex = 0;
    if (red[0] > 0.0) frexp(red[0], &ex);
    sc = ldexp(1.0, ex);
    if (threadIdx.x == 0) gsc[e] = (float)sc;
  }
  const long long g = e / epb;
  const int el = (int)(e - g * epb);
  for (int i = threadIdx.x; i < per_elem; i += blockDim.x) {
    const int c = i / np, q = i - c * np;
    long long idx;
    if (std::is_same<GT, float>::value || dim == 2) {
      idx = ((g * nc + c) * np + q) * epb + el;
    } else {  // 3D 16-bit: component pairs (2w, 2w + 1) in one 32-bit word
      idx = (((g * 3 + c / 2) * np + q) * epb + el) * 2 + (c & 1);
    }
    out[idx] = (GT)(float)(ge[i] / sc);
  }
}

}  // namespace hmg
