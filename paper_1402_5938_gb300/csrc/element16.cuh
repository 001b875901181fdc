// FP16 / BF16 apply of the mixed-precision V-cycle, y += alpha * A x with FP32 vectors, for
// orders p <= 7 (N = p+1 <= 8 nodes per direction).
//
// The 1D contractions of sum factorization (paper Sec. 2.3: interpolation B from the GLL
// nodes to the Gauss points and the GLL basis derivative Bd = D B there) run on the tensor
// cores as mma.sync m16n8k8 with 16-bit operands and FP32 accumulation: a contraction along
// one direction is the product (lines x N) * (N x N), so 16 lines of the element tile form
// the rows of one MMA, the N <= 8 input values its K and the N <= 8 outputs its columns.
// The gradient is taken with Bd directly, g_1 = (B x B x Bd) u and so on, so that the three
// components at a Gauss point come out of the last forward contraction in the same register
// positions: the pointwise product with the geometric factors G and the first transposed
// contraction then happen in registers (the accumulator layout of m16n8k8 equals its A-operand
// layout), and only four intermediate results per element travel through shared memory.
//
// Each warp owns a group of EW elements (EW * N^(d-1) >= 64 lines) and, after the block fills
// a table of index offsets once, needs no block-wide synchronization; a group's G slab arrives
// by one bulk TMA copy while its forward contractions run. FP16 uses power-of-two scales for x
// (per element group, largest entry in [0.5, 1)) and for G (per element, set at setup), which
// keep every intermediate far inside the FP16 range for N <= 8; BF16 needs none.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "element.cuh"

namespace hmg {

constexpr int kMaxN16 = 8;

// 1D tables [q][a] (Gauss point q, GLL node a) of one order, N <= 8.
struct Tab16 {
  float B[kMaxN16 * kMaxN16];
  float Bd[kMaxN16 * kMaxN16];
};

template <typename T>
struct Lowp;
template <>
struct Lowp<__half> {
  static constexpr bool kScaled = true;
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ uint16_t bits(float v) { return __half_as_ushort(__float2half_rn(v)); }
  static __device__ __forceinline__ float val(uint16_t b) { return __half2float(__ushort_as_half(b)); }
  static __device__ __forceinline__ float2 val2(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
  }
  static __device__ __forceinline__ void mma(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(b0));
  }
};
template <>
struct Lowp<__nv_bfloat16> {
  static constexpr bool kScaled = false;
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ uint16_t bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
  static __device__ __forceinline__ float val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
  static __device__ __forceinline__ float2 val2(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
  }
  static __device__ __forceinline__ void mma(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(b0));
  }
};

// Shared-memory layout of k_apply16 (every region starts on 16 bytes): a block-wide table of
// per-lane index offsets (the same for every element group), then one region per warp.
//
// A line buffer holds MT*16 rows of 8 16-bit values. Each row carries LPR = 8 / NPAD lines of
// up to NPAD values (NPAD = 2, 4 or 8, the smallest power of two >= N): line L sits in row
// L % H, slot L / H (H = 16 MT rows), value b at column slot * NPAD + b. The 1D tables enter the
// MMA block-diagonally (one NPAD x NPAD block per slot), so one m16n8k8 contracts 16 LPR lines.
template <int DIM, int N, int HALF = 0>
struct Apply16Cfg {
  static constexpr int NP = Sh<DIM, N>::NP, NL = Sh<DIM, N>::NL, NC = Sh<DIM, N>::NC;
  static constexpr int NPAD = N <= 2 ? 2 : (N <= 4 ? 4 : 8);
  static constexpr int LPR = 8 / NPAD;  // lines per MMA row
  // elements per warp group: >= 64 lines (HALF: about half of that, for meshes too small to give
  // every warp a group)
  static constexpr int EW0 = LPR == 1 ? (64 + NL - 1) / NL : (32 * LPR) / NL;
  static constexpr int EW1 = HALF ? (EW0 + 1) / 2 : EW0;
  static constexpr int EW = EW1 < 1 ? 1 : (EW1 > 32 ? 32 : EW1);
  static constexpr int NLG = EW * NL;                               // lines of a group along any direction
  static constexpr int MT = ((NLG + LPR - 1) / LPR + 15) / 16;      // 16-row MMA tiles
  static constexpr int H = MT * 16;
  static constexpr int BUF = MT * 16 * 8;        // 16-bit values per line buffer
  static constexpr int NB = DIM == 3 ? 6 : 4;    // line buffers
  static constexpr int VPL = (EW * NP + 31) / 32;  // gathered values per lane
  static constexpr int GSLAB = EW * NC * NP * 2;   // bytes of a group's factors
  static constexpr int GSLOT = (GSLAB + 16 + 15) / 16 * 16;
  static constexpr int al16(int b) { return (b + 15) / 16 * 16; }
  // block table, per (m-tile, lane) and accumulator entry u = 0..3 (row g / g+8, column 2t / 2t+1)
  static constexpr int TAB_S1 = 0;                         // short4: MAP-1 store offsets (-1: none)
  static constexpr int TAB_S2 = TAB_S1 + MT * 32 * 8;      // short4: MAP-2 store offsets (3D)
  static constexpr int TAB_G = TAB_S2 + MT * 32 * 8;       // short4: factor offsets (-1: no point)
  static constexpr int TAB_YO = TAB_G + MT * 32 * 8;       // int4: node offsets in the element
  static constexpr int TAB_YI = TAB_YO + MT * 32 * 16;     // int4: element | face bits << 8 (-1: none)
  static constexpr int TAB_GO = TAB_YI + MT * 32 * 16;     // gather: node offset in the element (-1: none)
  static constexpr int TAB_GC = TAB_GO + VPL * 32 * 4;     // gather: element | face bits << 8 | dest << 16
  static constexpr int TAB_BYTES = al16(TAB_GC + VPL * 32 * 4);
  // per warp
  static constexpr int OFF_BAR = 0;  // one mbarrier
  static constexpr int OFF_BUF = 16;
  static constexpr int OFF_G = OFF_BUF + NB * BUF * 2;
  static constexpr int OFF_BASE = OFF_G + GSLOT;
  static constexpr int OFF_FLAG = OFF_BASE + al16(EW * 8);
  static constexpr int OFF_FAC = OFF_FLAG + al16(EW * 4);
  static constexpr int WARP_BYTES = OFF_FAC + al16(EW * 4);
  static size_t smem(int warps) { return (size_t)TAB_BYTES + (size_t)warps * WARP_BYTES; }
  // buffer position of value b of line L
  __host__ __device__ static constexpr int pos(int L, int b) { return (L % H) * 8 + (L / H) * NPAD + b; }
};

namespace lp {

// A operand of one 16-row tile (rows 16 mt .. 16 mt + 15, 16 bytes each) by ldmatrix: lane l
// passes the address of row (l & 15) of the tile (ra = shared address of that row); a lane then
// holds rows g and g+8, columns 2t, 2t+1, the m16n8k8 A fragment. ldA2 loads the same rows of two
// buffers (lanes 16-31 address the second).
__device__ __forceinline__ void ldA(uint32_t ra, uint32_t& a0, uint32_t& a1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(a0), "=r"(a1) : "r"(ra) : "memory");
}
__device__ __forceinline__ void ldA2(uint32_t ra, uint32_t& a0, uint32_t& a1, uint32_t& b0, uint32_t& b1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(a0), "=r"(a1), "=r"(b0), "=r"(b1)
               : "r"(ra)
               : "memory");
}

// Store an accumulator tile into the line buffer of the next direction at the table's offsets
// (negative: padding entry, skipped).
template <typename T>
__device__ __forceinline__ void stC(uint16_t* buf, const float (&c)[4], short4 o) {
  if (o.x >= 0) buf[o.x] = Lowp<T>::bits(c[0]);
  if (o.y >= 0) buf[o.y] = Lowp<T>::bits(c[1]);
  if (o.z >= 0) buf[o.z] = Lowp<T>::bits(c[2]);
  if (o.w >= 0) buf[o.w] = Lowp<T>::bits(c[3]);
}

}  // namespace lp

template <int DIM, int N, typename T, int HALF>
__global__ void __launch_bounds__(256)
k_apply16(const float* __restrict__ x, float* __restrict__ y, const T* __restrict__ G16,
          const float* __restrict__ gsc, const Mesh m, const __grid_constant__ Tab16 tab, const float alpha,
          const long long ngroups, int* __restrict__ err) {
  using C = Apply16Cfg<DIM, N, HALF>;
  using L = Lowp<T>;
  constexpr int NP = C::NP, NL = C::NL, NC = C::NC, EW = C::EW, NLG = C::NLG, MT = C::MT, BUF = C::BUF;
  constexpr int H = C::H, NPAD = C::NPAD;
  extern __shared__ __align__(128) unsigned char smem16[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const long long nx = m.Nn[0], nxy = m.Nn[0] * m.Nn[1];

  // ---- block table of per-lane index offsets (depends on the lane and the mesh strides only) ----
  short4* ts1 = reinterpret_cast<short4*>(smem16 + C::TAB_S1);
  short4* ts2 = reinterpret_cast<short4*>(smem16 + C::TAB_S2);
  short4* tgo = reinterpret_cast<short4*>(smem16 + C::TAB_G);
  int4* tyo = reinterpret_cast<int4*>(smem16 + C::TAB_YO);
  int4* tyi = reinterpret_cast<int4*>(smem16 + C::TAB_YI);
  int* go = reinterpret_cast<int*>(smem16 + C::TAB_GO);
  int* gcode = reinterpret_cast<int*>(smem16 + C::TAB_GC);
  for (int i = threadIdx.x; i < MT * 32 * 4; i += blockDim.x) {
    const int mt = i >> 7, ln = (i >> 2) & 31, u = i & 3;
    const int r = mt * 16 + (ln >> 2) + 8 * (u >> 1);       // accumulator row
    const int col = 2 * (ln & 3) + (u & 1);                   // accumulator column
    const int L = (col / NPAD) * H + r, c = col % NPAD;       // line and its value index
    const bool ok = L < NLG && c < N;
    const int e = L / NL, rem = L % NL;
    // MAP 1: value c of line (s, b) -> value b of line (s, c); MAP 2 (3D): value c of line
    // (e, a, b) -> value a of line (e, c, b)
    const int s1 = ok ? C::pos((L / N) * N + c, L % N) : -1;
    const int s2 = (ok && DIM == 3) ? C::pos(((L / (N * N)) * N + c) * N + L % N, (L / N) % N) : -1;
    // factors: 3D point-major [e][q][6] (three 32-bit loads per point), 2D [e][3][q]
    const int gq = !ok ? -1 : (DIM == 3 ? (e * NP + c * NL + rem) * NC : e * NC * NP + c * NL + rem);
    const int kk = DIM == 3 ? rem / N : 0, jj = DIM == 3 ? rem % N : rem;
    int fb = (c == 0) | ((c == N - 1) << 1) | ((jj == 0) << 2) | ((jj == N - 1) << 3);
    if (DIM == 3) fb |= ((kk == 0) << 4) | ((kk == N - 1) << 5);
    reinterpret_cast<short*>(ts1)[i] = (short)s1;
    reinterpret_cast<short*>(ts2)[i] = (short)s2;
    reinterpret_cast<short*>(tgo)[i] = (short)gq;
    reinterpret_cast<int*>(tyo)[i] = ok ? (int)(kk * nxy + jj * nx + c) : 0;
    reinterpret_cast<int*>(tyi)[i] = ok ? (e | (fb << 8)) : -1;
  }
  for (int i = threadIdx.x; i < C::VPL * 32; i += blockDim.x) {
    const int e = i / NP, a = i - e * NP;
    const int ii = a % N, jj = (a / N) % N, kk = DIM == 3 ? a / (N * N) : 0;
    int fb = (ii == 0) | ((ii == N - 1) << 1) | ((jj == 0) << 2) | ((jj == N - 1) << 3);
    if (DIM == 3) fb |= ((kk == 0) << 4) | ((kk == N - 1) << 5);
    const bool ok = i < EW * NP;
    go[i] = ok ? (int)(kk * nxy + jj * nx + ii) : -1;
    gcode[i] = ok ? (e | (fb << 8) | (C::pos(e * NL + a / N, ii) << 16)) : 0;
  }

  unsigned char* ws = smem16 + C::TAB_BYTES + warp * C::WARP_BYTES;
  uint64_t* bar = reinterpret_cast<uint64_t*>(ws + C::OFF_BAR);
  uint16_t* buf = reinterpret_cast<uint16_t*>(ws + C::OFF_BUF);
  unsigned char* gslot = ws + C::OFF_G;
  long long* ebase = reinterpret_cast<long long*>(ws + C::OFF_BASE);
  int* eflag = reinterpret_cast<int*>(ws + C::OFF_FLAG);
  float* efac = reinterpret_cast<float*>(ws + C::OFF_FAC);

  // zero the line buffers and the factor slot once: padding rows and columns are never written
  // afterwards, and stale factors of a short last group stay finite
  for (int i = lane; i < C::NB * BUF / 2; i += 32) reinterpret_cast<uint32_t*>(buf)[i] = 0u;
  for (int i = lane; i < C::GSLOT / 4; i += 32) reinterpret_cast<uint32_t*>(gslot)[i] = 0u;
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();

  // B-operand fragments (k = 2t, 2t+1; n = g), block-diagonal with NPAD x NPAD blocks:
  // forward tables M[n][k], transposed M[k][n]
  auto tb = [&](const float* M, int q, int a) {
    return (q / NPAD == a / NPAD && q % NPAD < N && a % NPAD < N) ? M[(q % NPAD) * N + a % NPAD] : 0.0f;
  };
  const uint32_t fB = L::pack(tb(tab.B, g, 2 * t), tb(tab.B, g, 2 * t + 1));
  const uint32_t fD = L::pack(tb(tab.Bd, g, 2 * t), tb(tab.Bd, g, 2 * t + 1));
  const uint32_t bB = L::pack(tb(tab.B, 2 * t, g), tb(tab.B, 2 * t + 1, g));
  const uint32_t bD = L::pack(tb(tab.Bd, 2 * t, g), tb(tab.Bd, 2 * t + 1, g));
  // ldmatrix row address of this lane: row (lane & 15) of a tile, in the buffer of half-warp lane >> 4
  const uint32_t rowb = (uint32_t)(lane & 15) * 16u;

  const long long gstride = (long long)gridDim.x * (blockDim.x >> 5);
  long long grp = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  auto slab = [&](long long gi, const char** src, uint32_t* bytes) -> int {
    const long long e0 = gi * EW;
    const long long ne = min((long long)EW, m.nelem - e0);
    const char* p = reinterpret_cast<const char*>(G16 + e0 * NC * NP);
    const int off = (int)(reinterpret_cast<uintptr_t>(p) & 15);
    *src = p - off;
    *bytes = (uint32_t)((ne * NC * NP * 2 + off + 15) & ~15LL);
    return off;
  };

  uint32_t phase = 0u;
  for (; grp < ngroups; grp += gstride) {
    // this group's factors: one bulk copy into the warp's slot (last read before the previous
    // group's closing __syncwarp), waited for after the forward contractions
    const char* gsrc;
    uint32_t gbytes;
    const int goff = slab(grp, &gsrc, &gbytes);
    if (lane == 0) {
      fence_proxy_async_smem();
      bulk_g2s(gslot, gsrc, gbytes, bar);
    }
    const long long e0 = grp * EW;
    const int ne = (int)min((long long)EW, m.nelem - e0);
    if (lane < ne) elem_base(m, e0 + lane, &ebase[lane], &eflag[lane]);
    __syncwarp();

    // ---- gather x (boundary nodes read as 0) ----
    float xv[C::VPL];
#pragma unroll
    for (int u = 0; u < C::VPL; ++u) {
      const int o = go[u * 32 + lane], code = gcode[u * 32 + lane];
      const int e = code & 0xff;
      xv[u] = 0.0f;
      if (o >= 0 && e < ne && !((code >> 8) & 0xff & eflag[e])) xv[u] = x[ebase[e] + o];
    }
    // FP16: one power-of-two scale for the group (largest scaled |x| in [0.5, 1)), exact
    float sx = 1.0f;
    if (L::kScaled) {
      float amax = 0.0f;
#pragma unroll
      for (int u = 0; u < C::VPL; ++u) amax = fmaxf(amax, fabsf(xv[u]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      int ex = 0;
      if (amax > 0.0f) frexpf(amax, &ex);
      sx = ldexpf(1.0f, -ex);
    }
    if (lane < EW) efac[lane] = alpha * ((gsc != nullptr && lane < ne) ? gsc[e0 + lane] : 1.0f) / sx;
#pragma unroll
    for (int u = 0; u < C::VPL; ++u)
      if (u * 32 + lane < EW * NP) buf[gcode[u * 32 + lane] >> 16] = L::bits(xv[u] * sx);
    __syncwarp();

    const uint32_t s0 = smem_addr(buf);  // shared address of line buffer 0; buffer k at s0 + k * BUF * 2
    auto sa = [&](int k, int mt) { return s0 + (uint32_t)(k * BUF * 2 + mt * 256) + rowb; };
    auto sa2 = [&](int k0, int k1, int mt) {  // lanes 0-15 address buffer k0, lanes 16-31 buffer k1
      return s0 + (uint32_t)(((lane >> 4) ? k1 : k0) * BUF * 2 + mt * 256) + rowb;
    };
    uint16_t* B0 = buf;
    uint16_t* B1 = buf + BUF;
    uint16_t* B2 = buf + 2 * BUF;
    uint16_t* B3 = buf + 3 * BUF;
    uint16_t* B4 = buf + (DIM == 3 ? 4 : 0) * BUF;
    uint16_t* B5 = buf + (DIM == 3 ? 5 : 0) * BUF;
    // ---- forward: direction 0 (i): t1 = B x, t2 = Bd x -> direction-1 buffers B1, B2 ----
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      uint32_t a0, a1;
      lp::ldA(sa(0, mt), a0, a1);
      float c1[4] = {0.f, 0.f, 0.f, 0.f}, c2[4] = {0.f, 0.f, 0.f, 0.f};
      L::mma(c1, a0, a1, fB);
      L::mma(c2, a0, a1, fD);
      const short4 o = ts1[mt * 32 + lane];
      lp::stC<T>(B1, c1, o);
      lp::stC<T>(B2, c2, o);
    }
    __syncwarp();
    if (DIM == 3) {
      // direction 1 (j): t11 = B t1, t12 = Bd t1, t21 = B t2 -> direction-2 buffers B0, B3, B4
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        uint32_t a0, a1, p0, p1;
        lp::ldA2(sa2(1, 2, mt), a0, a1, p0, p1);
        float c11[4] = {0.f, 0.f, 0.f, 0.f}, c12[4] = {0.f, 0.f, 0.f, 0.f}, c21[4] = {0.f, 0.f, 0.f, 0.f};
        L::mma(c11, a0, a1, fB);
        L::mma(c12, a0, a1, fD);
        L::mma(c21, p0, p1, fB);
        const short4 o = ts2[mt * 32 + lane];
        lp::stC<T>(B0, c11, o);
        lp::stC<T>(B3, c12, o);
        lp::stC<T>(B4, c21, o);
      }
      __syncwarp();
    }

    // the factors (bounded wait; all lanes agree on the outcome)
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, phase, kWaitPolls));
    if (!ok) {
      if (lane == 0) atomicExch(err, kErrTmaTimeout);
      return;
    }
    phase ^= 1u;
    const uint16_t* Gs = reinterpret_cast<const uint16_t*>(gslot + goff);

    // ---- last forward direction, pointwise G, first transposed contraction (registers) ----
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      float gr[3][4];  // gradient components along directions 0, 1, 2 at this lane's 4 points
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int u = 0; u < 4; ++u) gr[d][u] = 0.0f;
      uint32_t a0, a1, p0, p1;
      if (DIM == 3) {
        lp::ldA2(sa2(0, 3, mt), a0, a1, p0, p1);
        L::mma(gr[2], a0, a1, fD);  // Bd_k B_j B_i x
        L::mma(gr[1], p0, p1, fB);  // B_k Bd_j B_i x
        lp::ldA(sa(4, mt), a0, a1);
        L::mma(gr[0], a0, a1, fB);  // B_k B_j Bd_i x
      } else {
        lp::ldA2(sa2(1, 2, mt), a0, a1, p0, p1);
        L::mma(gr[1], a0, a1, fD);  // Bd_j B_i x
        L::mma(gr[0], p0, p1, fB);  // B_j Bd_i x
      }
      // entries without a point read the first factors of the slot and get v = 0 (they meet
      // zero table entries in the next contraction, so they must be finite)
      const short4 go4 = tgo[mt * 32 + lane];
      const short gq[4] = {go4.x, go4.y, go4.z, go4.w};
      float v[3][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool pv = gq[u] >= 0;
        const uint16_t* q = Gs + (pv ? gq[u] : 0);
        if (DIM == 3) {
          const uint32_t* q32 = reinterpret_cast<const uint32_t*>(q);  // 4-byte aligned: 12 B per point
          const float2 ga = L::val2(q32[0]), gb = L::val2(q32[1]), gc = L::val2(q32[2]);
          const float g00 = ga.x, g01 = ga.y, g02 = gb.x, g11 = gb.y, g12 = gc.x, g22 = gc.y;
          v[0][u] = pv ? g00 * gr[0][u] + g01 * gr[1][u] + g02 * gr[2][u] : 0.0f;
          v[1][u] = pv ? g01 * gr[0][u] + g11 * gr[1][u] + g12 * gr[2][u] : 0.0f;
          v[2][u] = pv ? g02 * gr[0][u] + g12 * gr[1][u] + g22 * gr[2][u] : 0.0f;
        } else {
          const float g00 = L::val(q[0]), g01 = L::val(q[NP]), g11 = L::val(q[2 * NP]);
          v[0][u] = pv ? g00 * gr[0][u] + g01 * gr[1][u] : 0.0f;
          v[1][u] = pv ? g01 * gr[0][u] + g11 * gr[1][u] : 0.0f;
          v[2][u] = 0.0f;
        }
      }
      // accumulator -> A operand: the contraction runs over this tile's columns
      if (DIM == 3) {
        float s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f}, s3[4] = {0.f, 0.f, 0.f, 0.f};
        L::mma(s1, L::pack(v[0][0], v[0][1]), L::pack(v[0][2], v[0][3]), bB);
        L::mma(s2, L::pack(v[1][0], v[1][1]), L::pack(v[1][2], v[1][3]), bB);
        L::mma(s3, L::pack(v[2][0], v[2][1]), L::pack(v[2][2], v[2][3]), bD);
        const short4 o = ts2[mt * 32 + lane];
        lp::stC<T>(B1, s1, o);
        lp::stC<T>(B2, s2, o);
        lp::stC<T>(B5, s3, o);
      } else {
        float s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f};
        L::mma(s1, L::pack(v[0][0], v[0][1]), L::pack(v[0][2], v[0][3]), bB);
        L::mma(s2, L::pack(v[1][0], v[1][1]), L::pack(v[1][2], v[1][3]), bD);
        const short4 o = ts1[mt * 32 + lane];
        lp::stC<T>(B0, s1, o);
        lp::stC<T>(B3, s2, o);
      }
    }
    __syncwarp();

    if (DIM == 3) {
      // direction 1 transposed: s1' = B^T s1, r23 = Bd^T s2 + B^T s3 -> direction-0 buffers B0, B3
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        uint32_t a0, a1, p0, p1;
        float c1[4] = {0.f, 0.f, 0.f, 0.f}, c2[4] = {0.f, 0.f, 0.f, 0.f};
        lp::ldA2(sa2(1, 2, mt), a0, a1, p0, p1);
        L::mma(c1, a0, a1, bB);
        L::mma(c2, p0, p1, bD);
        lp::ldA(sa(5, mt), a0, a1);
        L::mma(c2, a0, a1, bB);
        const short4 o = ts1[mt * 32 + lane];
        lp::stC<T>(B0, c1, o);
        lp::stC<T>(B3, c2, o);
      }
      __syncwarp();
    }

    // ---- direction 0 transposed: y_e = Bd^T (.) + B^T (.), scatter-add to interior nodes ----
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      uint32_t a0, a1, p0, p1;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      lp::ldA2(sa2(0, 3, mt), a0, a1, p0, p1);
      L::mma(c, a0, a1, bD);
      L::mma(c, p0, p1, bB);
      const int4 yo = tyo[mt * 32 + lane], yi = tyi[mt * 32 + lane];
      const int off[4] = {yo.x, yo.y, yo.z, yo.w}, inf[4] = {yi.x, yi.y, yi.z, yi.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = inf[u] & 0xff;
        if (inf[u] >= 0 && e < ne && !((inf[u] >> 8) & eflag[e])) atomicAdd(y + ebase[e] + off[u], efac[e] * c[u]);
      }
    }
    __syncwarp();
  }
}

// 16-bit factors G16 = G / gsc[e] of one element per block, from G[e][c][q] (nc components, np
// points): point-major G16[e][q][c] when point_major (3D), else G16[e][c][q]. FP16 takes gsc[e] =
// the power of two with the element's largest |G| / gsc in [0.5, 1); BF16 gsc = nullptr (no scale).
template <typename T>
__global__ void k_pack_g16(const double* __restrict__ G, T* __restrict__ G16, float* __restrict__ gsc,
                           long long nelem, int nc, int np, int point_major) {
  const long long e = blockIdx.x;
  if (e >= nelem) return;
  const int per_elem = nc * np;
  const double* ge = G + e * per_elem;
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
  double sc = 1.0;
  if (gsc != nullptr) {
    int ex = 0;
    if (red[0] > 0.0) frexp(red[0], &ex);
    sc = ldexp(1.0, ex);
    if (threadIdx.x == 0) gsc[e] = (float)sc;
  }
  T* oe = G16 + e * per_elem;
  for (int i = threadIdx.x; i < per_elem; i += blockDim.x) {
    const int comp = i / np, q = i - comp * np;
    oe[point_major ? q * nc + comp : i] = (T)(float)(ge[i] / sc);
  }
}

}  // namespace hmg
