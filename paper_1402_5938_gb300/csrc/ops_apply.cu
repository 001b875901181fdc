// Instantiation and launch of the reduced-precision operator apply (pencil form, pencil.cuh; and
// for 16-bit factors at 3D orders 1-4 the tensor-core form, tc16.cuh) with FP32, FP16 or BF16
// geometric factors, the packing of those factors and the reference gradient table at setup.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdlib>
#include <vector>

#include "dispatch.cuh"
#include "ops.cuh"
#include "pencil.cuh"
#include "tc16.cuh"

namespace hmg {

namespace {

template <int DIM, typename GT>
cudaError_t apply_low_dim(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* G,
                          const float* gsc, float alpha, int variant, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    return launch_pencil<DIM, N, GT>(m, b, x, y, static_cast<const GT*>(G), gsc, alpha, variant, s);
  });
}

template <typename GT>
cudaError_t apply_low(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* G, const float* gsc,
                      float alpha, int variant, cudaStream_t s) {
  return m.dim == 3 ? apply_low_dim<3, GT>(m, b, x, y, G, gsc, alpha, variant, s)
                    : apply_low_dim<2, GT>(m, b, x, y, G, gsc, alpha, variant, s);
}

template <int N, typename GT>
cudaError_t launch_tc16_n(const Mesh& m, const float* x, float* y, const uint32_t* G, const float* gsc,
                          const void* phi, float alpha, float vsc, int* err, cudaStream_t s) {
  using C = Tc16Cfg<N>;
  const long long ntiles = tc16_tiles(m);
  if (ntiles == 0) return cudaSuccess;
  auto kern = k_apply_tc16<N, GT>;
  cudaError_t e = ensure_smem(kern, C::SMEM);
  if (e != cudaSuccess) return e;
  // co-resident CTAs share the SM's 512 tensor-memory columns: an allocation beyond them would
  // wait for another CTA to finish, so the shared-memory footprint must keep residency below that
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::THREADS, C::SMEM);
  if (e != cudaSuccess) return e;
  if (occ < 1 || occ * C::TMEM_COLS > 512) return cudaErrorInvalidConfiguration;
  const long long cap = (long long)device_sm_count() * occ;
  const long long grid = ntiles < cap ? ntiles : cap;
  kern<<<(unsigned)grid, C::THREADS, C::SMEM, s>>>(x, y, G, gsc, static_cast<const unsigned char*>(phi), m, alpha,
                                                  vsc, 1.0f / vsc, ntiles, err);
  return counted(cudaGetLastError());
}

template <typename GT>
cudaError_t launch_tc16(const Mesh& m, const float* x, float* y, const void* G, const float* gsc, const void* phi,
                        float alpha, float vsc, int* err, cudaStream_t s) {
  const uint32_t* g = static_cast<const uint32_t*>(G);
  switch (m.p + 1) {
    case 2: return launch_tc16_n<2, GT>(m, x, y, g, gsc, phi, alpha, vsc, err, s);
    case 3: return launch_tc16_n<3, GT>(m, x, y, g, gsc, phi, alpha, vsc, err, s);
    case 4: return launch_tc16_n<4, GT>(m, x, y, g, gsc, phi, alpha, vsc, err, s);
    case 5: return launch_tc16_n<5, GT>(m, x, y, g, gsc, phi, alpha, vsc, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool tc16_enabled() {
  static const bool on = [] {
    const char* v = getenv("HMG_TC16");
    return v && v[0] == '1';
  }();
  return on;
}

bool tc16_supported(const Mesh& m, int prec) {
  return tc16_enabled() && m.dim == 3 && m.p + 1 <= kTc16MaxN && (prec == HMG_PREC_FP16 || prec == HMG_PREC_BF16);
}

size_t tc16_factor_bytes(const Mesh& m) { return tc16_factor_words(m) * 4; }

cudaError_t launch_pack_tc16(const double* G, void* Gtc, float* gsc, const Mesh& m, int prec, cudaStream_t s) {
  if (m.nelem == 0) return cudaSuccess;
  if (!tc16_supported(m, prec)) return cudaErrorInvalidValue;
  const int nn = (m.p + 1) * (m.p + 1) * (m.p + 1), npad = (nn + 15) / 16 * 16;
  if (prec == HMG_PREC_FP16)
    k_pack_tc16<__half><<<(unsigned)m.nelem, 128, 0, s>>>(G, static_cast<uint32_t*>(Gtc), gsc, m, nn, npad);
  else
    k_pack_tc16<__nv_bfloat16><<<(unsigned)m.nelem, 128, 0, s>>>(G, static_cast<uint32_t*>(Gtc), gsc, m, nn, npad);
  return counted(cudaGetLastError());
}

size_t tc16_phi_bytes(const Mesh& m) {
  const int nn = (m.p + 1) * (m.p + 1) * (m.p + 1);
  const int npad = (nn + 15) / 16 * 16;
  return (size_t)3 * npad * npad * 2;
}

// Phi[node][c][q] = d phi_node / d xi_c at Gauss point q: the product of the 1D tables
// B[q][a] = l_a(g_q) and Bd = D B (the basis derivative at the Gauss points) along the three axes,
// node = i + n j + n^2 k, q = a + n b + n^2 c'. Written in FP16 at byte tc_core_off(c * NPAD + q,
// node, NPAD * 16); vsc is the power of two that keeps |v| = |G~ grad u~| <= 3 max_{c,q}
// sum_node |Phi| (|G~|, |x~| < 1) below 2^13.
void tc16_phi_image(const Basis1D& b, std::vector<unsigned char>& img, float* vsc) {
  const int n = b.n, nn = n * n * n, npad = (nn + 15) / 16 * 16, row = npad * 16;
  img.assign((size_t)3 * npad * npad * 2, 0);
  double cmax = 0.0;
  for (int c = 0; c < 3; ++c)
    for (int q = 0; q < nn; ++q) {
      const int qa[3] = {q % n, (q / n) % n, q / (n * n)};
      double rs = 0.0;
      for (int nd = 0; nd < nn; ++nd) {
        const int ia[3] = {nd % n, (nd / n) % n, nd / (n * n)};
        double v = 1.0;
        for (int a = 0; a < 3; ++a) v *= (a == c ? b.Bd : b.B)[qa[a] * n + ia[a]];
        rs += std::fabs(v);
        const __half h = __float2half_rn((float)v);
        *reinterpret_cast<__half*>(&img[tc_core_off(c * npad + q, nd, row)]) = h;
      }
      cmax = std::max(cmax, rs);
    }
  int ex = 0;
  std::frexp(3.0 * cmax, &ex);  // 3 cmax < 2^ex
  *vsc = std::ldexp(1.0f, 13 - ex);
}

size_t low_factor_bytes(const Mesh& m, int prec) {
  return pencil_factor_values(m.dim, m.p + 1, m.nelem) * (prec == HMG_PREC_FP32 ? 4 : 2);
}

cudaError_t launch_apply_low(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* G,
                             const float* gsc, float alpha, int prec, cudaStream_t s, int variant,
                             const Tc16Data* tc, int* err) {
  if (variant == kApplyLowTc) {
    if (!tc || !tc->G || !tc->phi || !err || !gsc || !tc16_supported(m, prec)) return cudaErrorInvalidValue;
    if (prec == HMG_PREC_FP16) return launch_tc16<__half>(m, x, y, tc->G, gsc, tc->phi, alpha, tc->vsc, err, s);
    return launch_tc16<__nv_bfloat16>(m, x, y, tc->G, gsc, tc->phi, alpha, tc->vsc, err, s);
  }
  if (prec == HMG_PREC_FP32) return apply_low<float>(m, b, x, y, G, nullptr, alpha, variant, s);
  if (prec == HMG_PREC_FP16) return apply_low<__half>(m, b, x, y, G, gsc, alpha, variant, s);
  if (prec == HMG_PREC_BF16) return apply_low<__nv_bfloat16>(m, b, x, y, G, gsc, alpha, variant, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_pack_low(const double* G, void* Glow, float* gsc, const Mesh& m, int prec, cudaStream_t s) {
  if (m.nelem == 0) return cudaSuccess;
  const int np = (int)(m.dim == 3 ? (long long)(m.p + 1) * (m.p + 1) * (m.p + 1) : (long long)(m.p + 1) * (m.p + 1));
  const int epb = pencil_shape(m.dim, m.p + 1).epb;
  if (prec == HMG_PREC_FP32)
    k_pack_grouped<float><<<(unsigned)m.nelem, 128, 0, s>>>(G, static_cast<float*>(Glow), nullptr, m.nelem, m.dim,
                                                            np, epb);
  else if (prec == HMG_PREC_FP16)
    k_pack_grouped<__half><<<(unsigned)m.nelem, 128, 0, s>>>(G, static_cast<__half*>(Glow), gsc, m.nelem, m.dim,
                                                             np, epb);
  else if (prec == HMG_PREC_BF16)
    k_pack_grouped<__nv_bfloat16><<<(unsigned)m.nelem, 128, 0, s>>>(G, static_cast<__nv_bfloat16*>(Glow), gsc,
                                                                     m.nelem, m.dim, np, epb);
  else
    return cudaErrorInvalidValue;
  return counted(cudaGetLastError());
}

}  // namespace hmg
