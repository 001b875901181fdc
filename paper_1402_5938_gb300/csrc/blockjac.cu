// Element-block Jacobi smoother (paper Sec. 3.2.3 and Sec. 4.4, Table 7): the exact inverses of
// the element matrices on each element's interior nodes, point Jacobi on the nodes that elements
// share (faces, edges, vertices).
//
// Blocks: Kb holds, per element, the MI x MI block (MI = (p-1)^d) of K_e on the element-interior
// local nodes, x fastest; k_block_invert replaces it in place by its inverse. An element-interior
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

// x_I(e) += omega * Kinv_e src_I(e) for EPC elements per thread block, TPE threads per element.
// Kinv_e is read column by column (Kb[(e * MI + c) * MI + r]), consecutive threads on
// consecutive rows r (coalesced).
template <int DIM>
__global__ void __launch_bounds__(256)
k_block_smooth(const double* __restrict__ Kb, const double* __restrict__ src, double* __restrict__ x,
               const Mesh m, const int MI, const int tpe, const double omega) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int epc = blockDim.x / tpe;
  const int le = threadIdx.x / tpe, lt = threadIdx.x - le * tpe;
  double* sv = reinterpret_cast<double*>(smem_raw) + le * MI;
  const long long e = (long long)blockIdx.x * epc + le;
  const bool live = le < epc && e < m.nelem;
  if (live)
    for (int r = lt; r < MI; r += tpe) sv[r] = src[interior_node<DIM>(m, e, r)];
  __syncthreads();
  if (!live) return;
  const double* K = Kb + e * (long long)MI * MI;
  for (int r = lt; r < MI; r += tpe) {
    double z0 = 0.0, z1 = 0.0;  // two independent chains
    int c = 0;
    for (; c + 1 < MI; c += 2) {
      z0 = fma(K[(long long)c * MI + r], sv[c], z0);
      z1 = fma(K[(long long)(c + 1) * MI + r], sv[c + 1], z1);
    }
    if (c < MI) z0 = fma(K[(long long)c * MI + r], sv[c], z0);
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

cudaError_t launch_block_smooth(const Mesh& m, const double* Kb, const double* src, double* x, double omega,
                                cudaStream_t s) {
  const int MI = block_size_of(m);
  if (MI <= 0) return cudaSuccess;
  int tpe = ((MI + 31) / 32) * 32;
  if (tpe > 256) tpe = 256;
  const int epc = 256 / tpe;
  const long long blocks = (m.nelem + epc - 1) / epc;
  const size_t smem = (size_t)epc * MI * sizeof(double);
  if (smem > 48 * 1024) return cudaErrorInvalidValue;  // MI <= 1000 gives <= 8 KB per element
  if (m.dim == 3) k_block_smooth<3><<<(unsigned)blocks, epc * tpe, smem, s>>>(Kb, src, x, m, MI, tpe, omega);
  else k_block_smooth<2><<<(unsigned)blocks, epc * tpe, smem, s>>>(Kb, src, x, m, MI, tpe, omega);
  return counted(cudaGetLastError());
}

cudaError_t launch_mask_elem_interior(double* dinv, const Mesh& m, cudaStream_t s) {
  if (m.p < 2) return cudaSuccess;
  long long g = (m.N + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  k_mask_elem_interior<<<(unsigned)g, 256, 0, s>>>(dinv, m);
  return counted(cudaGetLastError());
}

}  // namespace hmg
