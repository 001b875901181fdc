// Element-block Jacobi smoother (paper Sec. 3.2.3 and Sec. 4.4, Table 7): the exact inverses of
// the element matrices on each element's interior nodes, point Jacobi on the nodes that elements
// share (faces, edges, vertices).
//
// Blocks: Kb holds, per element, the MI x MI block (MI = (p-1)^d) of K_e on the element-interior
// local nodes, x fastest; k_block_invert replaces it in place by its inverse, and k_block_pack
// lays the inverses out for the smoother's 16-byte loads (Kp). An element-interior
// node belongs to that element alone, so the block is the assembled operator's block as well,
// and the blocks of different elements touch disjoint unknowns: the smoother's update
//   x_I(e) += omega * Kb_e^-1 r_I(e)   (every element),   x_s += omega * r_s / a_ss   (shared s)
// needs no atomics and no weighting.
#include "common.cuh"
#include "ops.cuh"

namespace hmg {
namespace {

// In-place Gauss-Jordan inversion of one MI x MI block per thread block (no pivoting: the
// blocks are symmetric positive definite). Step k stages row k and column k in shared memory,
// then every entry is updated in place:
//   a_kk <- 1/a_kk,  a_kj <- a_kj/a_kk,  a_ik <- -a_ik/a_kk,  a_ij <- a_ij - a_ik a_kj / a_kk.
// A pivot that is not positive and finite leaves the block as it is and sets *bad.
__global__ void __launch_bounds__(512) k_block_invert(double* __restrict__ Kb, const int MI, int* __restrict__ bad) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* rowk = reinterpret_cast<double*>(smem_raw);
  double* colk = rowk + MI;
  double* A = Kb + (long long)blockIdx.x * MI * MI;
  const int tot = MI * MI;
  for (int k = 0; k < MI; ++k) {
    for (int j = threadIdx.x; j < MI; j += blockDim.x) {
      rowk[j] = A[k * MI + j];
      colk[j] = A[j * MI + k];
    }
    __syncthreads();
    const double piv = rowk[k];
    if (!(piv > 0.0) || !isfinite(piv)) {  // same shared value in every thread: a uniform exit
      if (threadIdx.x == 0) atomicExch(bad, 1);
      return;
    }
    const double ip = 1.0 / piv;
    for (int t = threadIdx.x; t < tot; t += blockDim.x) {
      const int i = t / MI, j = t - i * MI;
      double v;
      if (i == k && j == k) v = ip;
      else if (i == k) v = rowk[j] * ip;
      else if (j == k) v = -colk[i] * ip;
      else v = fma(-colk[i] * ip, rowk[j], A[t]);
      A[t] = v;
    }
    __syncthreads();
  }
}

// Global node of the r-th element-interior local node (x fastest over (p-1)^DIM) of element e.
template <int DIM>
__device__ __forceinline__ long long interior_node(const Mesh& m, long long e, int r) {
  const int M = m.p - 1;
  const int i = r % M + 1, j = (r / M) % M + 1;
  const long long ex = e % m.E[0], r1 = e / m.E[0];
  if (DIM == 3) {
    const int k = r / (M * M) + 1;
    const long long ey = r1 % m.E[1], ez = r1 / m.E[1];
    return ((ez * m.p + k) * m.Nn[1] + ey * m.p + j) * m.Nn[0] + ex * m.p + i;
  }
  return (r1 * m.p + j) * m.Nn[0] + ex * m.p + i;
}

// Repack the inverses for the smoother: column pairs interleaved per row,
//   Kp[((e * C2 + c2) * MI + r) * 2 + h] = Kinv_e[r][2 c2 + h]   (C2 = ceil(MI/2), 0 past MI),
// so that one 16-byte load per thread gives two entries of a row and consecutive threads
// (rows) read consecutive 16-byte pairs. Kb holds the Gauss-Jordan result, whose [c][r]
// entry (column-major reading) is Kinv_e[r][c].
__global__ void k_block_pack(const double* __restrict__ Kb, double* __restrict__ Kp, const long long nelem,
                             const int MI) {
  const int C2 = (MI + 1) / 2;
  const long long tot = nelem * C2 * MI * 2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int h = (int)(t & 1);
    const long long q = t >> 1;
    const int r = (int)(q % MI);
    const long long q2 = q / MI;
    const int c2 = (int)(q2 % C2);
    const long long e = q2 / C2;
    const int col = 2 * c2 + h;
    Kp[t] = col < MI ? Kb[(e * MI + col) * MI + r] : 0.0;
  }
}

// x_I(e) += omega * Kinv_e src_I(e) for `epc` consecutive elements per thread block: src on
// their interior nodes is staged in shared memory (zero-padded to an even length), then the
// block's threads walk the flattened (element, row) pairs, each a dot product over the row's
// column pairs with 16-byte loads of Kp and of the staged vector.
template <int DIM>
__global__ void __launch_bounds__(1024)
k_block_smooth(const double* __restrict__ Kp, const double* __restrict__ src, double* __restrict__ x,
               const Mesh m, const int MI, const int epc, const double omega) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int C2 = (MI + 1) / 2, MIp = 2 * C2;
  double* sv = reinterpret_cast<double*>(smem_raw);
  const long long e0 = (long long)blockIdx.x * epc;
  const int ne = (int)min((long long)epc, m.nelem - e0);
  for (int t = threadIdx.x; t < ne * MIp; t += blockDim.x) {
    const int le = t / MIp, r = t - le * MIp;
    sv[t] = r < MI ? src[interior_node<DIM>(m, e0 + le, r)] : 0.0;
  }
  __syncthreads();
  const double2* K2 = reinterpret_cast<const double2*>(Kp);
  for (int t = threadIdx.x; t < ne * MI; t += blockDim.x) {
    const int le = t / MI, r = t - le * MI;
    const long long e = e0 + le;
    const double2* Kr = K2 + e * (long long)C2 * MI + r;  // pair c2 of row r at Kr[c2 * MI]
    const double2* s2 = reinterpret_cast<const double2*>(sv + le * MIp);
    double z0 = 0.0, z1 = 0.0;
#pragma unroll 4
    for (int c2 = 0; c2 < C2; ++c2) {
      const double2 k = Kr[(long long)c2 * MI];
      const double2 v = s2[c2];
      z0 = fma(k.x, v.x, z0);
      z1 = fma(k.y, v.y, z1);
    }
    const long long g = interior_node<DIM>(m, e, r);
    x[g] = fma(omega, z0 + z1, x[g]);
  }
}

// dinv[g] = 0 at element-interior nodes (every axis index not a multiple of p).
__global__ void k_mask_elem_interior(double* __restrict__ dinv, const Mesh m) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < m.N; g += (long long)gridDim.x * blockDim.x) {
    const long long I = g % m.Nn[0], rr = g / m.Nn[0];
    const long long J = rr % m.Nn[1], K = rr / m.Nn[1];
    bool inner = (I % m.p != 0) && (J % m.p != 0);
    if (m.dim == 3) inner = inner && (K % m.p != 0);
    if (inner) dinv[g] = 0.0;
  }
}

}  // namespace

int block_size_of(const Mesh& m) {
  if (m.p < 2) return 0;
  int s = 1;
  for (int a = 0; a < m.dim; ++a) s *= m.p - 1;
  return s;
}

cudaError_t launch_block_invert(double* Kb, long long nelem, int MI, int* bad, cudaStream_t s) {
  if (MI <= 0 || nelem <= 0) return cudaSuccess;
  const int threads = MI * MI >= 4096 ? 512 : 256;
  const size_t smem = 2 * (size_t)MI * sizeof(double);
  k_block_invert<<<(unsigned)nelem, threads, smem, s>>>(Kb, MI, bad);
  return counted(cudaGetLastError());
}

long long packed_block_doubles(long long nelem, int MI) { return nelem * ((MI + 1) / 2) * MI * 2; }

cudaError_t launch_block_pack(const double* Kb, double* Kp, long long nelem, int MI, cudaStream_t s) {
  if (MI <= 0 || nelem <= 0) return cudaSuccess;
  long long g = (packed_block_doubles(nelem, MI) + 255) / 256;
  if (g > (long long)device_sm_count() * 32) g = (long long)device_sm_count() * 32;
  k_block_pack<<<(unsigned)g, 256, 0, s>>>(Kb, Kp, nelem, MI);
  return counted(cudaGetLastError());
}

cudaError_t launch_block_smooth(const Mesh& m, const double* Kp, const double* src, double* x, double omega,
                                cudaStream_t s) {
  const int MI = block_size_of(m);
  if (MI <= 0) return cudaSuccess;
  const int epc = MI >= 256 ? 1 : 256 / MI;  // about 256 rows per block
  int threads = ((epc * MI + 31) / 32) * 32;
  if (threads > 1024) threads = 1024;
  const long long blocks = (m.nelem + epc - 1) / epc;
  const size_t smem = (size_t)epc * (2 * ((MI + 1) / 2)) * sizeof(double);  // <= 8 KB
  if (m.dim == 3) k_block_smooth<3><<<(unsigned)blocks, threads, smem, s>>>(Kp, src, x, m, MI, epc, omega);
  else k_block_smooth<2><<<(unsigned)blocks, threads, smem, s>>>(Kp, src, x, m, MI, epc, omega);
  return counted(cudaGetLastError());
}

cudaError_t launch_mask_elem_interior(double* dinv, const Mesh& m, cudaStream_t s) {
  if (m.p < 2) return cudaSuccess;
  long long g = (m.N + 255) / 256;
  if (g > (long long)device_sm_count() * 16) g = (long long)device_sm_count() * 16;
  k_mask_elem_interior<<<(unsigned)g, 256, 0, s>>>(dinv, m);
  return counted(cudaGetLastError());
}

}  // namespace hmg
