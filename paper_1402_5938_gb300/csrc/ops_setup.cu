// Instantiation and launch of the setup-time element kernels: geometric factors,
// operator diagonal, load vector, dense coarsest operator.
#include "dispatch.cuh"
#include "ops.cuh"

namespace hmg {

namespace {

template <int DIM>
cudaError_t geom_stage_dim(const Mesh& m, const Basis1D& b, double amp, const double* coords, double* Js,
                           cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    const size_t per = (size_t)(1 + DIM) * NP * sizeof(double);
    const int epb = epb_for(per);
    auto k1 = k_geom_stage<DIM, N>;
    cudaError_t e = ensure_smem(k1, per * epb);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem + epb - 1) / epb;
    k1<<<(unsigned)blocks, 256, per * epb, s>>>(Js, m, amp, coords, make_geotab<N>(b), epb);
    return counted(cudaGetLastError());
  });
}

template <int DIM>
cudaError_t geom_point_dim(const Mesh& m, const Basis1D& b, double mu_a, double mu_b, double mu_k,
                           const double* mu_arr, const double* Js, double* G, double* wdetJ, int* bad,
                           cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    const long long tot = m.nelem * NP;
    const unsigned g2 = (unsigned)std::min<long long>((tot + 255) / 256, (long long)device_sm_count() * 64);
    k_geom_point<DIM, N><<<g2, 256, 0, s>>>(Js, G, wdetJ, m, mu_a, mu_b, mu_k, mu_arr, make_geotab<N>(b), bad);
    return counted(cudaGetLastError());
  });
}

template <int DIM>
cudaError_t extract_xq_dim(const Mesh& m, const Basis1D& b, const double* Js, double* xq, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    const long long tot = m.nelem * Sh<DIM, N>::NP;
    const unsigned g = (unsigned)std::min<long long>((tot + 255) / 256, (long long)device_sm_count() * 64);
    k_extract_xq<DIM, N><<<g, 256, 0, s>>>(Js, xq, m);
    return counted(cudaGetLastError());
  });
}

template <int DIM>
cudaError_t diag_dim(const Mesh& m, const Basis1D& b, const double* G, double* diag, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    const size_t per = 2 * NP * sizeof(double);
    const int epb = epb_for(per);
    auto k = k_diag<DIM, N>;
    cudaError_t e = ensure_smem(k, per * epb);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem + epb - 1) / epb;
    k<<<(unsigned)blocks, 256, per * epb, s>>>(G, diag, m, make_geotab<N>(b), epb);
    return counted(cudaGetLastError());
  });
}

template <int DIM>
cudaError_t mass_dim(const Mesh& m, const Basis1D& b, const double* f, double* out,
                     const double* wdetJ, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    const size_t per = NP * sizeof(double);
    const int epb = epb_for(per);
    auto k = k_mass<DIM, N>;
    cudaError_t e = ensure_smem(k, per * epb);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem + epb - 1) / epb;
    k<<<(unsigned)blocks, 256, per * epb, s>>>(f, out, wdetJ, m, make_geotab<N>(b), epb);
    return counted(cudaGetLastError());
  });
}

template <int DIM>
cudaError_t dense_dim(const Mesh& m, const Basis1D& b, const double* G, double* A, long long nI,
                      double* Ke, double* Kb, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    constexpr long long MI = DIM == 3 ? (N - 2) * (N - 2) * (N - 2) : (N - 2) * (N - 2);
    const long long ncol = Kb != nullptr ? MI : NP;
    if (ncol == 0) return cudaSuccess;
    const size_t per = (size_t)(1 + DIM) * NP * sizeof(double);
    const int epb = epb_for(per);
    auto k = k_elem_dense<DIM, N>;
    cudaError_t e = ensure_smem(k, per * epb);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem * ncol + epb - 1) / epb;
    k<<<(unsigned)blocks, 256, per * epb, s>>>(G, A, m, make_tab<N, double>(b), nI, epb, Ke, Kb);
    return counted(cudaGetLastError());
  });
}

}  // namespace

cudaError_t launch_geom_stage(const Mesh& m, const Basis1D& b, double amp, const double* coords, double* Js,
                              cudaStream_t s) {
  return m.dim == 3 ? geom_stage_dim<3>(m, b, amp, coords, Js, s) : geom_stage_dim<2>(m, b, amp, coords, Js, s);
}

cudaError_t launch_geom_point(const Mesh& m, const Basis1D& b, double mu_a, double mu_b, double mu_k,
                              const double* mu_arr, const double* Js, double* G, double* wdetJ, int* bad,
                              cudaStream_t s) {
  return m.dim == 3 ? geom_point_dim<3>(m, b, mu_a, mu_b, mu_k, mu_arr, Js, G, wdetJ, bad, s)
                    : geom_point_dim<2>(m, b, mu_a, mu_b, mu_k, mu_arr, Js, G, wdetJ, bad, s);
}

cudaError_t launch_extract_xq(const Mesh& m, const Basis1D& b, const double* Js, double* xq, cudaStream_t s) {
  return m.dim == 3 ? extract_xq_dim<3>(m, b, Js, xq, s) : extract_xq_dim<2>(m, b, Js, xq, s);
}

cudaError_t launch_level_coords(const Mesh& m0, const Basis1D& b0, const double* X0, const Mesh& mk,
                                const Basis1D& bk, double* Xk, cudaStream_t s) {
  MapNodes nodes{};
  for (int i = 0; i < b0.n; ++i) nodes.r0[i] = b0.r[i];
  for (int i = 0; i < bk.n; ++i) nodes.rk[i] = bk.r[i];
  const unsigned g = (unsigned)std::min<long long>((mk.N + 255) / 256, (long long)device_sm_count() * 64);
  if (mk.N == 0) return cudaSuccess;
  if (m0.dim == 3)
    k_level_coords<3><<<g, 256, 0, s>>>(X0, m0, mk, nodes, Xk);
  else
    k_level_coords<2><<<g, 256, 0, s>>>(X0, m0, mk, nodes, Xk);
  return counted(cudaGetLastError());
}

cudaError_t launch_diag(const Mesh& m, const Basis1D& b, const double* G, double* diag, cudaStream_t s) {
  return m.dim == 3 ? diag_dim<3>(m, b, G, diag, s) : diag_dim<2>(m, b, G, diag, s);
}

cudaError_t launch_mass(const Mesh& m, const Basis1D& b, const double* f, double* out,
                        const double* wdetJ, cudaStream_t s) {
  return m.dim == 3 ? mass_dim<3>(m, b, f, out, wdetJ, s) : mass_dim<2>(m, b, f, out, wdetJ, s);
}

cudaError_t launch_elem_dense(const Mesh& m, const Basis1D& b, const double* G, double* A,
                              long long nI, cudaStream_t s) {
  return m.dim == 3 ? dense_dim<3>(m, b, G, A, nI, nullptr, nullptr, s)
                    : dense_dim<2>(m, b, G, A, nI, nullptr, nullptr, s);
}

cudaError_t launch_elem_mats(const Mesh& m, const Basis1D& b, const double* G, double* Ke, cudaStream_t s) {
  return m.dim == 3 ? dense_dim<3>(m, b, G, nullptr, 0, Ke, nullptr, s)
                    : dense_dim<2>(m, b, G, nullptr, 0, Ke, nullptr, s);
}

cudaError_t launch_elem_blocks(const Mesh& m, const Basis1D& b, const double* G, double* Kb, cudaStream_t s) {
  return m.dim == 3 ? dense_dim<3>(m, b, G, nullptr, 0, nullptr, Kb, s)
                    : dense_dim<2>(m, b, G, nullptr, 0, nullptr, Kb, s);
}

}  // namespace hmg
