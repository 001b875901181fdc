// Reduced-precision operator apply of the mixed V-cycle on the fifth-generation tensor cores
// (tcgen05), 3D orders 1-4: y += alpha * A x with FP32 vectors, geometric factors stored in 16
// bits (paper Sec. 2.3: the matrix-free apply, (A_k)_ij = sum_e sum_q (grad phi_i)^T G_q
// (grad phi_j) with G_q = mu w det J J^-1 J^-T at the Gauss points).
//
// At these orders an element's reference gradient matrix Phi (n^3 nodes x 3 n^3 Gauss-point
// derivatives: dphi_node/dxi_c at point q, the tensor product of the 1D interpolation and
// differentiation tables) is small enough to stay in shared memory (96 KB at order 4), so the
// element work becomes two dense products over a tile of 128 elements instead of twelve 1D
// passes:
//   grad u [128 x 3 n^3] = X [128 x n^3] Phi                 (tensor cores, FP32 in tensor memory)
//   v_q = G_q grad u_q at every Gauss point                    (CUDA cores, FP32)
//   y_e [128 x n^3]  = V [128 x 3 n^3] Phi^T                  (tensor cores, FP32 in tensor memory)
// then scatter-add into y. The tensor-core work (4 x 128 x 3 n^6 flops per tile, 2.5x-11x the
// sum-factorized count) is cheap next to the memory traffic: the 12 bytes of factors per Gauss
// point (read coalesced, one tile ahead in L2) and the tile's nodes.
//
// A tile is a block of 8 x 4 x 4 elements. Its nodes form a box of (8p+1) x (4p+1) x (4p+1)
// nodes that is gathered once, row by row (consecutive lanes, consecutive nodes), into shared
// memory, from where each element takes its n^3 values: element-wise loads touch 16 sectors per
// warp access and cost several times more. The element results are added into y with one atomic
// per element node.
//
// Operands of the products are FP16: each element's nodal values are divided by a power of two
// (largest |x| / s_x in [0.5, 1)), the factors are stored divided by a per-element power of two
// (largest |G| / s_G in [0.5, 1); FP16 or BF16 storage), v is multiplied by a fixed power of two
// that keeps it well inside the FP16 range; products accumulate in FP32 and the scales are undone
// when y is scattered. Per output this adds to the FP32 pencil form's error about four FP16
// roundings (x, Phi twice, v) relative to sum_e |Phi|^T |G| |Phi| |x|.
//
// Warp roles, persistent CTA over tiles t = blockIdx.x + k gridDim.x, the three element stages
// working on different tiles at once:
//   warps 0-3   gather: thread = element (warp = z-layer of the block); the box of tile i into
//               shared memory, then (once MMA 1 of tile i-1 has read X) X, and the scales into a ring
//   warps 4-11  pointwise: warp w reads tensor-memory lanes 32 (w mod 4) .. + 31 (the tile's
//               elements); warps w and w + 4 take 8 of each chunk's 16 points; v into a 4-slot ring
//   warps 12-15 scatter: thread = element; y_e from tensor memory, atomics into y
//   warp 16     allocates tensor memory; one thread copies Phi, prefetches the next tile's
//               factors into L2 and issues the MMAs
// Every wait on an mbarrier is bounded; on a timeout the kernel sets the error flag and the
// remaining waits return at once, so the CTA finishes (with wrong values) and frees its tensor
// memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "element.cuh"
#include "umma.cuh"

namespace hmg {

template <int N>
struct Tc16Cfg {
  static constexpr int P = N - 1;
  static constexpr int NN = N * N * N;                // nodes (= Gauss points) per element
  static constexpr int NPAD = (NN + 15) / 16 * 16;    // padded to the MMA's K step
  static constexpr int M = 128;                       // elements per tile (MMA rows)
  static constexpr int TBX = 8, TBY = 4, TBZ = 4;     // the tile's block of elements
  static constexpr int BX = TBX * P + 1, BY = TBY * P + 1, BZ = TBZ * P + 1;  // its node box
  static constexpr int BOX = BX * BY * BZ;
  static constexpr int NCH = NPAD / 16;               // 16-point chunks per tile
  static constexpr int CORE_ROW = NPAD * 16;          // bytes between 8-row core-matrix groups
  static constexpr int PHI_BYTES = 3 * NPAD * NPAD * 2;
  static constexpr int X_BYTES = M * NPAD * 2;
  static constexpr int SLAB = M * 16 * 2;             // one component of one chunk of V
  static constexpr int VSLOT = 3 * SLAB;
  static constexpr int NVS = 4;
  static constexpr int NSX = 4;                       // ring of per-element x scales (gather -> scatter)
  static constexpr int GCHUNK_WORDS = 3 * 16 * M;     // factor words of one chunk: [w][q][element]
  static constexpr int OFF_X = PHI_BYTES;
  static constexpr int OFF_V = OFF_X + X_BYTES;
  static constexpr int OFF_BOX = OFF_V + NVS * VSLOT;
  static constexpr int OFF_MISC = OFF_BOX + (BOX * 4 + 15) / 16 * 16;
  static constexpr int NBAR = 8 + 2 * NVS + 2 * NSX;
  static constexpr int SMEM = OFF_MISC + NBAR * 8 + 16 + NSX * M * 4;
  static constexpr int TMEM_COLS = 4 * NPAD <= 32 ? 32 : 4 * NPAD <= 64 ? 64 : 4 * NPAD <= 128 ? 128 : 4 * NPAD <= 256 ? 256 : 512;
  static constexpr int THREADS = 17 * 32;
  static_assert(TBX * TBY * TBZ == M, "tile block");
  static_assert(BX <= 64, "a box row is read by two loads per lane");
  static_assert(4 * NPAD <= 512, "grad u and y of a tile must fit tensor memory");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Tiles of a level's mesh (blocks of 8 x 4 x 4 elements, the last ones of each axis partial).
inline long long tc16_tiles(const Mesh& m) {
  return (long long)((m.E[0] + 7) / 8) * ((m.E[1] + 3) / 4) * ((m.E[2] + 3) / 4);
}
// Words of the tensor-core factor layout of a level: per tile and chunk of 16 Gauss points,
// [component pair w][point][element slot] (32-bit words holding two 16-bit factors).
inline size_t tc16_factor_words(const Mesh& m) {
  const int n = m.p + 1, nn = n * n * n, npad = (nn + 15) / 16 * 16;
  return (size_t)tc16_tiles(m) * npad * 3 * 128;
}

// Byte offset of entry (row, col) of a no-swizzle operand whose 16-byte core rows run along col:
// core matrix (row / 8, col / 8) at (row / 8) * row_stride + (col / 8) * 128.
__host__ __device__ constexpr int tc_core_off(int row, int col, int row_stride) {
  return (row / 8) * row_stride + (col / 8) * 128 + (row % 8) * 16 + (col % 8) * 2;
}

// One try_wait with a suspend-time hint: a waiting thread sleeps in hardware until the phase
// completes or about `ns` nanoseconds pass, instead of spinning on issue slots the working warps need.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
      : "memory");
  return done != 0;
}
// Bounded wait (at most about kTcWaitTries * 100 us); after the first timeout in the CTA (*abort
// set) every wait returns at once.
constexpr uint32_t kTcWaitTries = 20000;
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort, int* err) {
  for (uint32_t it = 0; it < kTcWaitTries; ++it) {
    if (mbar_try(bar, parity, 100000u)) return true;
    if (*abort) return false;
  }
  *abort = 1;
  atomicExch(err, kErrTmaTimeout);
  return false;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Power of two s with m / s in [0.5, 1) (1 for m = 0), and 1 / s, from the exponent field.
__device__ __forceinline__ void pow2_scale(float m, float& s, float& inv) {
  const int e = (int)((__float_as_uint(m) >> 23) & 0xffu);
  if (m == 0.0f) {
    s = 1.0f;
    inv = 1.0f;
    return;
  }
  const int ee = e == 0 ? 1 : e;  // subnormal maxima: scale as for the smallest normal exponent
  s = __uint_as_float((uint32_t)(ee + 1) << 23);
  inv = __uint_as_float((uint32_t)(253 - ee) << 23);
}

// Element e of mesh m: first global node, face bits (x-, x+, y-, y+, z-, z+).
__device__ __forceinline__ void tc_elem(const Mesh& m, long long e, long long& nb, int& fl) {
  const int ex = (int)(e % m.E[0]);
  const long long r = e / m.E[0];
  const int ey = (int)(r % m.E[1]);
  const int ez = (int)(r / m.E[1]);
  nb = ((long long)ez * m.p * m.Nn[1] + (long long)ey * m.p) * m.Nn[0] + (long long)ex * m.p;
  fl = (ex == 0) | ((ex == m.E[0] - 1) << 1) | ((ey == 0) << 2) | ((ey == m.E[1] - 1) << 3) | ((ez == 0) << 4) |
       ((ez == m.E[2] - 1) << 5);
}
template <int N>
__device__ __forceinline__ bool tc_node_bd(int nd, int fl) {
  const int i = nd % N, j = (nd / N) % N, k = nd / (N * N);
  return ((i == 0) & (fl & 1)) | ((i == N - 1) & ((fl >> 1) & 1)) | ((j == 0) & ((fl >> 2) & 1)) |
         ((j == N - 1) & ((fl >> 3) & 1)) | ((k == 0) & ((fl >> 4) & 1)) | ((k == N - 1) & ((fl >> 5) & 1));
}
// Offset of local node nd from the element's first node (nx, nxy: node strides along y and z;
// a level's node count is below 2^31).
template <int N>
__device__ __forceinline__ int tc_node_off(int nd, int nx, int nxy) {
  const int i = nd % N, j = (nd / N) % N, k = nd / (N * N);
  return i + j * nx + k * nxy;
}

template <typename GT>
__device__ __forceinline__ float2 unpack16(uint32_t u) {
  if constexpr (std::is_same<GT, __half>::value) return __half22float2(*reinterpret_cast<const __half2*>(&u));
  else return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
}
__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ void box_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// First element (ex0, ey0, ez0) of tile t of mesh m (tiles x fastest).
__device__ __forceinline__ void tc_tile_origin(const Mesh& m, long long t, int& ex0, int& ey0, int& ez0) {
  const int ntx = (m.E[0] + 7) / 8, nty = (m.E[1] + 3) / 4;
  ex0 = (int)(t % ntx) * 8;
  const long long r = t / ntx;
  ey0 = (int)(r % nty) * 4;
  ez0 = (int)(r / nty) * 4;
}

// G: the level's 16-bit factors in the tensor-core layout (tc16_factor_words words); gsc[e] the
// element's factor scale; phi: the Phi image (PHI_BYTES, core-matrix order, rows c * NPAD + q,
// columns nodes); vsc / vinv: the power of two applied to v and its inverse; ntiles =
// tc16_tiles(m).
template <int N, typename GT>
__global__ void __launch_bounds__(Tc16Cfg<N>::THREADS, 1)
k_apply_tc16(const float* __restrict__ x, float* __restrict__ y, const uint32_t* __restrict__ G,
             const float* __restrict__ gsc, const unsigned char* __restrict__ phi, const Mesh m, const float alpha,
             const float vsc, const float vinv, const long long ntiles, int* __restrict__ err) {
  using C = Tc16Cfg<N>;
  constexpr int NN = C::NN, NPAD = C::NPAD, NCH = C::NCH, P = C::P, BX = C::BX, BY = C::BY;
  extern __shared__ __align__(1024) unsigned char sm_tc[];
  unsigned char* sPhi = sm_tc;
  unsigned char* sX = sm_tc + C::OFF_X;
  unsigned char* sV = sm_tc + C::OFF_V;
  float* sBox = reinterpret_cast<float*>(sm_tc + C::OFF_BOX);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm_tc + C::OFF_MISC);
  uint64_t* phi_full = bars + 0;
  uint64_t* x_full = bars + 1;
  uint64_t* d1_full = bars + 2;
  uint64_t* d1_empty = bars + 3;
  uint64_t* d2_full = bars + 4;
  uint64_t* d2_empty = bars + 5;
  uint64_t* fin = bars + 6;
  uint64_t* v_full = bars + 8;
  uint64_t* v_empty = v_full + C::NVS;
  uint64_t* sx_full = v_empty + C::NVS;
  uint64_t* sx_empty = sx_full + C::NSX;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + C::NBAR);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  float* sxs = reinterpret_cast<float*>(tslot + 4);  // [NSX][128] x scales of tiles in flight

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    // arrival counts: per warp of the arriving role (gather 4, pointwise 8, scatter 4), else one
    // (the copy's expect_tx or an MMA commit)
    for (int b = 0; b < C::NBAR; ++b) {
      uint64_t* p = bars + b;
      int cnt = 1;
      if (p == x_full || p == d2_empty || (p >= sx_full && p < sx_full + 2 * C::NSX)) cnt = 4;
      if (p == d1_empty || (p >= v_full && p < v_full + C::NVS)) cnt = 8;
      mbar_init(p, cnt);
    }
    *abort = 0;
    mbar_init_fence();
  }
  if (warp == 16) {
    tmem_alloc(tslot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const long long nx = m.Nn[0], nxy = m.Nn[0] * m.Nn[1];

  if (warp < 4 || (warp >= 12 && warp < 16)) {
    // element of this thread: (lx, ly, lz) of the block, tensor-memory lane el
    const int el = (warp & 3) * 32 + lane;
    const int lx = el & 7, ly = (el >> 3) & 3, lz = el >> 5;
    struct Elem {
      long long e, nb;
      bool valid;
      int fl;
    };
    auto elem = [&](long long t) {
      Elem q;
      int ex0, ey0, ez0;
      tc_tile_origin(m, t, ex0, ey0, ez0);
      const int ex = ex0 + lx, ey = ey0 + ly, ez = ez0 + lz;
      q.valid = ex < m.E[0] && ey < m.E[1] && ez < m.E[2];
      q.e = q.valid ? ((long long)ez * m.E[1] + ey) * m.E[0] + ex : 0;
      q.nb = q.valid ? ((long long)ez * P * m.Nn[1] + (long long)ey * P) * m.Nn[0] + (long long)ex * P : 0;
      q.fl = (ex == 0) | ((ex == m.E[0] - 1) << 1) | ((ey == 0) << 2) | ((ey == m.E[1] - 1) << 3) | ((ez == 0) << 4) |
             ((ez == m.E[2] - 1) << 5);
      return q;
    };
    if (warp < 4) {
      // ---- gather: the tile's box by rows into shared memory (asynchronous 4-byte copies, lanes
      // along the row), then each element's values into X (FP16 at the element's power-of-two
      // scale: each 8-node core row stored at the scale of the running maximum, rows stored at a
      // smaller scale then multiplied by the exact power of two that brings them to the final one)
      const int eoff = (lz * P * BY + ly * P) * BX + lx * P;  // element's first node in the box
      constexpr int ROWS = NPAD / 8;
      int i = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        int ex0, ey0, ez0;
        tc_tile_origin(m, t, ex0, ey0, ez0);
        const long long gx0 = (long long)ex0 * P, gy0 = (long long)ey0 * P, gz0 = (long long)ez0 * P;
        const int bx = (int)(m.Nn[0] - gx0 < BX ? m.Nn[0] - gx0 : BX);
        const int by = (int)(m.Nn[1] - gy0 < BY ? m.Nn[1] - gy0 : BY);
        const int bz = (int)(m.Nn[2] - gz0 < C::BZ ? m.Nn[2] - gz0 : C::BZ);
        const float* xb = x + gz0 * nxy + gy0 * nx + gx0;
        // rows in rounds of 8 per warp, all loads of a round in flight before the stores
        const int nrows = by * bz;
        for (int r0 = warp * 8; r0 < nrows; r0 += 32) {
          float a[8], b[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int r = r0 + q, ry = r % by, rz = r / by;
            const float* src = xb + rz * nxy + ry * nx;
            a[q] = (r < nrows && lane < bx) ? __ldg(src + lane) : 0.0f;
            b[q] = (r < nrows && lane + 32 < bx) ? __ldg(src + lane + 32) : 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int r = r0 + q, ry = r % by, rz = r / by;
            float* dst = sBox + (rz * BY + ry) * BX;
            if (r < nrows && lane < bx) dst[lane] = a[q];
            if (r < nrows && lane + 32 < bx) dst[lane + 32] = b[q];
          }
        }
        box_sync();
        const Elem q = elem(t);
        if (i > 0) tc_wait(d1_full, (uint32_t)((i - 1) & 1), abort, err);  // X read by the last product
        const int sl = i % C::NSX;
        if (i >= C::NSX) tc_wait(sx_empty + sl, (uint32_t)((i / C::NSX - 1) & 1), abort, err);
        const float* eb = sBox + eoff;
        float mx = 0.0f;
        uint32_t ex[(ROWS + 3) / 4] = {};  // exponent field of each row's scale, 8 bits per row
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          float xr[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int nd = r * 8 + k;
            const int off = (nd % N) + ((nd / N) % N) * BX + (nd / (N * N)) * BX * BY;
            xr[k] = (nd < NN && q.valid && !tc_node_bd<N>(nd, q.fl)) ? eb[off] : 0.0f;
            mx = fmaxf(mx, fabsf(xr[k]));
          }
          float s, inv;
          pow2_scale(mx, s, inv);
          if (mx > 0.0f) ex[r / 4] |= ((__float_as_uint(s) >> 23) & 0xffu) << (8 * (r % 4));
          *reinterpret_cast<uint4*>(sX + tc_core_off(el, r * 8, C::CORE_ROW)) =
              make_uint4(pack_h2(xr[0] * inv, xr[1] * inv), pack_h2(xr[2] * inv, xr[3] * inv),
                         pack_h2(xr[4] * inv, xr[5] * inv), pack_h2(xr[6] * inv, xr[7] * inv));
        }
        float s, inv;
        pow2_scale(mx, s, inv);
        sxs[sl * C::M + el] = s;
        const int es = (int)((__float_as_uint(s) >> 23) & 0xffu);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int er = (int)((ex[r / 4] >> (8 * (r % 4))) & 0xffu), d = es - er;
          if (er != 0 && d > 0) {  // multiply by 2^-d (exact for results in the normal range; 0 if d > 24)
            uint4* p = reinterpret_cast<uint4*>(sX + tc_core_off(el, r * 8, C::CORE_ROW));
            const __half2 f = __float2half2_rn(d > 24 ? 0.0f : __uint_as_float((uint32_t)(127 - d) << 23));
            uint4 u = *p;
            __half2* hv = reinterpret_cast<__half2*>(&u);
#pragma unroll
            for (int w = 0; w < 4; ++w) hv[w] = __hmul2(hv[w], f);
            *p = u;
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(x_full);
          mbar_arrive(sx_full + sl);
        }
        box_sync();  // every element has read the box
      }
    } else {
      // ---- scatter: y_e * (alpha s_x s_G / vsc) from tensor memory, one atomic per element node
      const uint32_t tl = tbase + ((uint32_t)(lz * 32) << 16) + 3 * NPAD;
      int i = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const Elem q = elem(t);
        const int sl = i % C::NSX;
        tc_wait(sx_full + sl, (uint32_t)((i / C::NSX) & 1), abort, err);
        const float sc = q.valid ? alpha * sxs[sl * C::M + el] * gsc[q.e] * vinv : 0.0f;
        __syncwarp();
        if (lane == 0) mbar_arrive(sx_empty + sl);
        tc_wait(d2_full, (uint32_t)(i & 1), abort, err);
        __syncwarp();
        tc_fence_after();
        float* ye = y + q.nb;
#pragma unroll
        for (int k0 = 0; k0 < NPAD; k0 += 16) {
          float yv[16];
          tmem_ld16(tl + k0, yv);
          tmem_wait_ld();
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int nd = k0 + k;
            if (nd < NN && q.valid && !tc_node_bd<N>(nd, q.fl))
              atomicAdd(ye + (nd % N) + ((nd / N) % N) * nx + (nd / (N * N)) * nxy, sc * yv[k]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(d2_empty);
      }
    }
  } else if (warp < 12) {
    // ---- pointwise: v = G grad u at this thread's 8 points of each chunk; the factors of the next
    // chunk are loaded while this one is computed
    const int qd = warp & 3, h = (warp - 4) >> 2;
    const int el = qd * 32 + lane;
    const int lx = el & 7, ly = (el >> 3) & 3, lz = el >> 5;
    const uint32_t tl = tbase + ((uint32_t)(qd * 32) << 16);
    long long cs = 0;
    int i = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      int ex0, ey0, ez0;
      tc_tile_origin(m, t, ex0, ey0, ez0);
      const bool valid = ex0 + lx < m.E[0] && ey0 + ly < m.E[1] && ez0 + lz < m.E[2];
      const uint32_t* gt = G + (size_t)t * NCH * C::GCHUNK_WORDS + 8 * h * C::M + el;
      uint32_t gn[24];
#pragma unroll
      for (int w = 0; w < 3; ++w)
#pragma unroll
        for (int k = 0; k < 8; ++k) gn[w * 8 + k] = __ldg(gt + w * 16 * C::M + k * C::M);
      tc_wait(d1_full, (uint32_t)(i & 1), abort, err);
      __syncwarp();
      tc_fence_after();
#pragma unroll 1
      for (int j = 0; j < NCH; ++j, ++cs) {
        const int s = (int)(cs % C::NVS);
        const int q0 = 16 * j + 8 * h;
        uint32_t gc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) gc[k] = gn[k];
        if (j + 1 < NCH) {
          const uint32_t* gj = gt + (size_t)(j + 1) * C::GCHUNK_WORDS;
#pragma unroll
          for (int w = 0; w < 3; ++w)
#pragma unroll
            for (int k = 0; k < 8; ++k) gn[w * 8 + k] = __ldg(gj + w * 16 * C::M + k * C::M);
        }
        float ux[8], uy[8], uz[8];
        tmem_ld8(tl + 0 * NPAD + q0, ux);
        tmem_ld8(tl + 1 * NPAD + q0, uy);
        tmem_ld8(tl + 2 * NPAD + q0, uz);
        tmem_wait_ld();
        if (cs >= C::NVS) tc_wait(v_empty + s, (uint32_t)((cs / C::NVS - 1) & 1), abort, err);
        __syncwarp();
        // v overwrites grad u in place: (g00, g01) (g02, g11) (g12, g22)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          float v0 = 0.0f, v1 = 0.0f, v2 = 0.0f;
          if (valid && q0 + k < NN) {
            const float2 a = unpack16<GT>(gc[k]);
            const float2 b = unpack16<GT>(gc[8 + k]);
            const float2 c = unpack16<GT>(gc[16 + k]);
            v0 = vsc * (a.x * ux[k] + a.y * uy[k] + b.x * uz[k]);
            v1 = vsc * (a.y * ux[k] + b.y * uy[k] + c.x * uz[k]);
            v2 = vsc * (b.x * ux[k] + c.x * uy[k] + c.y * uz[k]);
          }
          ux[k] = v0;
          uy[k] = v1;
          uz[k] = v2;
        }
        unsigned char* vs = sV + s * C::VSLOT + tc_core_off(el, 8 * h, 256);
        *reinterpret_cast<uint4*>(vs) = make_uint4(pack_h2(ux[0], ux[1]), pack_h2(ux[2], ux[3]),
                                                   pack_h2(ux[4], ux[5]), pack_h2(ux[6], ux[7]));
        *reinterpret_cast<uint4*>(vs + C::SLAB) = make_uint4(pack_h2(uy[0], uy[1]), pack_h2(uy[2], uy[3]),
                                                             pack_h2(uy[4], uy[5]), pack_h2(uy[6], uy[7]));
        *reinterpret_cast<uint4*>(vs + 2 * C::SLAB) = make_uint4(pack_h2(uz[0], uz[1]), pack_h2(uz[2], uz[3]),
                                                                 pack_h2(uz[4], uz[5]), pack_h2(uz[6], uz[7]));
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(v_full + s);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(d1_empty);
    }
  } else {
    // ---- warp 16: Phi, L2 prefetches of the factors one tile ahead, MMA issue (one thread)
    if (lane == 0) {
      constexpr uint32_t ID = idesc_f16(128, NPAD, false, false);
      constexpr uint32_t ID_T = idesc_f16(128, NPAD, false, true);
      constexpr uint32_t TILE_BYTES = (uint32_t)NCH * C::GCHUNK_WORDS * 4;
      const unsigned char* Gb = reinterpret_cast<const unsigned char*>(G);
      auto prefetch_tile = [&](long long tp) {
        for (uint32_t o = 0; o < TILE_BYTES; o += 65536)
          prefetch_l2_bulk(Gb + tp * TILE_BYTES + o, TILE_BYTES - o < 65536 ? TILE_BYTES - o : 65536);
      };
      mbar_expect_tx(phi_full, C::PHI_BYTES);
      for (int off = 0; off < C::PHI_BYTES; off += 16384) {
        const int nb = C::PHI_BYTES - off < 16384 ? C::PHI_BYTES - off : 16384;
        bulk_copy_g2s(sPhi + off, phi + off, (uint32_t)nb, phi_full);
      }
      if (blockIdx.x < ntiles) prefetch_tile(blockIdx.x);
      const uint32_t aX = smem_addr(sX), aV = smem_addr(sV), aPhi = smem_addr(sPhi);
      tc_wait(phi_full, 0, abort, err);
      long long cs = 0;
      int i = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        if (t + gridDim.x < ntiles) prefetch_tile(t + gridDim.x);
        tc_wait(x_full, (uint32_t)(i & 1), abort, err);
        if (i > 0) tc_wait(d1_empty, (uint32_t)((i - 1) & 1), abort, err);
        tc_fence_after();
        // grad u = X Phi: K = nodes (16 per step), one N = NPAD product per component
        for (int ks = 0; ks < NPAD / 16; ++ks) {
          const uint64_t ad = sdesc(aX + ks * 256, 128, C::CORE_ROW);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const uint64_t bd = sdesc(aPhi + c * (NPAD / 8) * C::CORE_ROW + ks * 256, 128, C::CORE_ROW);
            mma_f16(tbase + c * NPAD, ad, bd, ID, ks > 0);
          }
        }
        mma_commit(d1_full);
        // y_e = V Phi^T: K = (component, point), 16 points per chunk; Phi read MN-major
        for (int j = 0; j < NCH; ++j, ++cs) {
          const int s = (int)(cs % C::NVS);
          tc_wait(v_full + s, (uint32_t)((cs / C::NVS) & 1), abort, err);
          if (j == 0 && i > 0) tc_wait(d2_empty, (uint32_t)((i - 1) & 1), abort, err);
          tc_fence_after();
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const uint64_t ad = sdesc(aV + s * C::VSLOT + c * C::SLAB, 128, 256);
            const uint64_t bd = sdesc(aPhi + (c * (NPAD / 8) + 2 * j) * C::CORE_ROW, C::CORE_ROW, 128);
            mma_f16(tbase + 3 * NPAD, ad, bd, ID_T, !(j == 0 && c == 0));
          }
          mma_commit(v_empty + s);
        }
        mma_commit(d2_full);
      }
      mma_commit(fin);
      tc_wait(fin, 0, abort, err);
    }
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 16) {
    tc_fence_after();
    tmem_dealloc(tbase, C::TMEM_COLS);
  }
}

// Factors of element e (one block per element) from G[e][c][q] (FP64) into the tensor-core layout:
// divided by gsc[e], the power of two that puts the element's largest |G| / gsc in [0.5, 1)
// (written here), as component pairs (g00, g01) (g02, g11) (g12, g22) in 32-bit words at the
// element's tile and slot. The buffer is zero-filled beforehand, so padding points and slots stay
// zero.
template <typename GT>
__global__ void k_pack_tc16(const double* __restrict__ G, uint32_t* __restrict__ out, float* __restrict__ gsc,
                            const Mesh m, int nn, int npad) {
  const long long e = blockIdx.x;
  if (e >= m.nelem) return;
  const double* ge = G + e * 6 * nn;
  __shared__ double red[32];
  double amax = 0.0;
  for (int i = threadIdx.x; i < 6 * nn; i += blockDim.x) amax = fmax(amax, fabs(ge[i]));
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
  const double sc = ldexp(1.0, ex);
  if (threadIdx.x == 0) gsc[e] = (float)sc;
  const int x = (int)(e % m.E[0]);
  const long long r = e / m.E[0];
  const int yy = (int)(r % m.E[1]), z = (int)(r / m.E[1]);
  const int ntx = (m.E[0] + 7) / 8, nty = (m.E[1] + 3) / 4;
  const long long t = ((long long)(z / 4) * nty + yy / 4) * ntx + x / 8;
  const int el = (x % 8) + 8 * (yy % 4) + 32 * (z % 4);
  for (int i = threadIdx.x; i < 3 * nn; i += blockDim.x) {
    const int w = i / nn, q = i % nn, j = q / 16, ql = q % 16;
    const GT lo = (GT)(float)(ge[(2 * w) * nn + q] / sc), hi = (GT)(float)(ge[(2 * w + 1) * nn + q] / sc);
    uint16_t lb, hb;
    memcpy(&lb, &lo, 2);
    memcpy(&hb, &hi, 2);
    out[(((t * (npad / 16) + j) * 3 + w) * 16 + ql) * 128 + el] = (uint32_t)lb | ((uint32_t)hb << 16);
  }
}

}  // namespace hmg
