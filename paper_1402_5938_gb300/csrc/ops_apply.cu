// Instantiation and launch of the reduced-precision operator apply (pencil form, pencil.cuh) with
// FP32, FP16 or BF16 geometric factors, and the packing of those factors at setup.
#include "dispatch.cuh"
#include "ops.cuh"
#include "pencil.cuh"

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

}  // namespace

size_t low_factor_bytes(const Mesh& m, int prec) {
  return pencil_factor_values(m.dim, m.p + 1, m.nelem) * (prec == HMG_PREC_FP32 ? 4 : 2);
}

cudaError_t launch_apply_low(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* G,
                             const float* gsc, float alpha, int prec, cudaStream_t s, int variant) {
  if (prec == HMG_PREC_FP32) return apply_low<float>(m, b, x, y, G, nullptr, alpha, variant, s);
  if (prec == HMG_PREC_FP16) return apply_low<__half>(m, b, x, y, G, gsc, alpha, variant, s);
  if (prec == HMG_PREC_BF16) return apply_low<__nv_bfloat16>(m, b, x, y, G, nullptr, alpha, variant, s);
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
    k_pack_grouped<__nv_bfloat16><<<(unsigned)m.nelem, 128, 0, s>>>(G, static_cast<__nv_bfloat16*>(Glow), nullptr,
                                                                     m.nelem, m.dim, np, epb);
  else
    return cudaErrorInvalidValue;
  return counted(cudaGetLastError());
}

}  // namespace hmg
