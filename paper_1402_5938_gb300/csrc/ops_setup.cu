// Instantiation and launch of the setup-time element kernels: geometric factors,
// operator diagonal, load vector, dense coarsest operator.
#include "dispatch.cuh"
#include "ops.cuh"

namespace hmg {

namespace {

template <int DIM>
cudaError_t geometry_dim(const Mesh& m, const Basis1D& b, double amp, double mu_a, double mu_b,
                         double mu_k, double* Js, double* G, double* wdetJ, int* bad, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    const GeoTab<N> tab = make_geotab<N>(b);
    const size_t per = (size_t)(1 + DIM) * NP * sizeof(double);
    const int epb = epb_for(per);
    auto k1 = k_geom_stage<DIM, N>;
    cudaError_t e = ensure_smem(k1, per * epb);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem + epb - 1) / epb;
    k1<<<(unsigned)blocks, 256, per * epb, s>>>(Js, m, amp, tab, epb);
    if ((e = counted(cudaGetLastError())) != cudaSuccess) return e;
    const long long tot = m.nelem * NP;
    const unsigned g2 = (unsigned)std::min<long long>((tot + 255) / 256, 152LL * 64);
    k_geom_point<DIM, N><<<g2, 256, 0, s>>>(Js, G, wdetJ, m, mu_a, mu_b, mu_k, tab, bad);
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
                      cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    const size_t per = (size_t)(1 + DIM) * NP * sizeof(double);
    const int epb = epb_for(per);
    auto k = k_elem_dense<DIM, N>;
    cudaError_t e = ensure_smem(k, per * epb);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem * NP + epb - 1) / epb;
    k<<<(unsigned)blocks, 256, per * epb, s>>>(G, A, m, make_tab<N, double>(b), nI, epb);
    return counted(cudaGetLastError());
  });
}

}  // namespace

cudaError_t launch_geometry(const Mesh& m, const Basis1D& b, double amp, double mu_a, double mu_b,
                            double mu_k, double* Js, double* G, double* wdetJ, int* bad, cudaStream_t s) {
  return m.dim == 3 ? geometry_dim<3>(m, b, amp, mu_a, mu_b, mu_k, Js, G, wdetJ, bad, s)
                    : geometry_dim<2>(m, b, amp, mu_a, mu_b, mu_k, Js, G, wdetJ, bad, s);
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
  return m.dim == 3 ? dense_dim<3>(m, b, G, A, nI, s) : dense_dim<2>(m, b, G, A, nI, s);
}

}  // namespace hmg
