// C ABI of libhmg: hierarchy setup and the multigrid / PCG drivers. Every step of the
// numerical path runs in this library's CUDA kernels; the host only sequences launches
// on the caller's stream and reads back one residual norm per iteration.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <map>
#include <tuple>
#include <type_traits>
#include <mutex>
#include <set>
#include <new>
#include <string>
#include <vector>

#include <chrono>
#include <cstdio>
#include <cstdlib>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "ops.cuh"
#include "problem.cuh"
#include "vector.cuh"

namespace hmg {

namespace {
thread_local std::string g_err;
}
void set_error(const std::string& msg) { g_err = msg; }

namespace {
std::atomic<long long> g_launches{0};
}
long long add_launches(long long n) { return g_launches.fetch_add(n) + n; }

int device_sm_count() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cached[dev].load();
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
    cached[dev].store(n);
  }
  return n;
}

namespace {
std::mutex g_smem_mu;
std::set<std::pair<const void*, int>> g_smem_done;
}
cudaError_t ensure_smem_ptr(const void* kernel, size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_smem_mu);
  if (g_smem_done.count({kernel, dev})) return cudaSuccess;
  (void)bytes;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) g_smem_done.insert({kernel, dev});
  return e;
}

// Phase tracing: an NVTX range per phase (visible to Nsight tools), and with HMG_TRACE=1 in the
// environment the phase's wall time (after synchronizing its stream) on stderr.
struct Phase {
  const char* name;
  cudaStream_t s;
  std::chrono::steady_clock::time_point t0;
  static bool timing() {
    static const bool on = [] {
      const char* v = getenv("HMG_TRACE");
      return v && v[0] == '1';
    }();
    return on;
  }
  Phase(const char* n, cudaStream_t st) : name(n), s(st) {
    nvtxRangePushA(n);
    if (timing()) {
      cudaStreamSynchronize(s);
      t0 = std::chrono::steady_clock::now();
    }
  }
  ~Phase() {
    if (timing()) {
      cudaStreamSynchronize(s);
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      fprintf(stderr, "hmg %s: %.3f ms\n", name, ms);
    }
    nvtxRangePop();
  }
};

}  // namespace hmg



using namespace hmg;

#define TRY(expr)                                                            \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) {                                                 \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));         \
      return _e == cudaErrorMemoryAllocation ? HMG_ENOMEM : HMG_EDEVICE;     \
    }                                                                        \
  } while (0)

#define CHECK(expr)                        \
  do {                                     \
    hmg_status _s = (expr);                \
    if (_s != HMG_OK) return _s;           \
  } while (0)

namespace {

Mesh make_mesh(int dim, const int E[3], int p) {
  Mesh m{};
  m.dim = dim;
  m.p = p;
  m.nelem = 1;
  m.N = 1;
  for (int a = 0; a < 3; ++a) {
    m.E[a] = a < dim ? E[a] : 1;
    m.Nn[a] = a < dim ? (long long)E[a] * p + 1 : 1;
    m.nelem *= m.E[a];
    m.N *= m.Nn[a];
  }
  return m;
}

long long interior_count(const Mesh& m) {
  long long n = 1;
  for (int a = 0; a < m.dim; ++a) n *= std::max(0LL, m.Nn[a] - 2);
  return n;
}

int nc_of(int dim) { return dim == 3 ? 6 : 3; }
long long np_of(const Mesh& m) { return m.dim == 3 ? (long long)(m.p + 1) * (m.p + 1) * (m.p + 1) : (long long)(m.p + 1) * (m.p + 1); }

// (nelem, p) of every level, finest first.
hmg_status level_shapes(const hmg_desc& d, std::vector<std::pair<std::vector<int>, int>>& out) {
  std::vector<int> E(d.nelem, d.nelem + 3);
  int p = d.order;
  out.clear();
  out.push_back({E, p});
  if (d.hier == HMG_HIER_P) {
    while (p > 1) {
      p = std::max(1, p / 2);
      out.push_back({E, p});
    }
  } else if (d.hier != HMG_HIER_H) {
    set_error("hier must be HMG_HIER_H or HMG_HIER_P");
    return HMG_EINVAL;
  }
  for (int k = 1; k < d.n_hlevels; ++k) {
    for (int a = 0; a < d.dim; ++a) {
      if (E[a] % 2) {
        set_error("mesh cannot be halved n_hlevels-1 times (odd element count)");
        return HMG_EINVAL;
      }
      E[a] /= 2;
    }
    out.push_back({E, p});
  }
  return HMG_OK;
}

// Largest element-interior block of the block Jacobi smoother ((p-1)^d unknowns: 3D p <= 11).
constexpr long long kMaxBlock = 1000;

hmg_status validate(const hmg_desc* d) {
  if (!d) { set_error("null descriptor"); return HMG_EINVAL; }
  if (d->dim != 2 && d->dim != 3) { set_error("dim must be 2 or 3"); return HMG_EINVAL; }
  if (d->order < 1 || d->order > 16) { set_error("order must be in 1..16"); return HMG_EINVAL; }
  for (int a = 0; a < d->dim; ++a)
    if (d->nelem[a] < 1 || d->nelem[a] > (1 << 20)) { set_error("nelem out of range"); return HMG_EINVAL; }
  if (d->n_hlevels < 1 || d->n_hlevels > 30) { set_error("n_hlevels must be >= 1"); return HMG_EINVAL; }
  {  // kernels index elements and nodes of a level with 32-bit integers
    long long ne = 1, nn = 1;
    for (int a = 0; a < d->dim; ++a) {
      ne *= d->nelem[a];
      nn *= (long long)d->nelem[a] * d->order + 1;
    }
    if (ne >= (1ll << 31) || nn >= (1ll << 31)) { set_error("more than 2^31 - 1 elements or nodes"); return HMG_EINVAL; }
  }
  if (d->smoother != HMG_SMOOTH_JACOBI && d->smoother != HMG_SMOOTH_CHEB && d->smoother != HMG_SMOOTH_L1JACOBI &&
      d->smoother != HMG_SMOOTH_BLOCKJACOBI) {
    set_error("bad smoother");
    return HMG_EINVAL;
  }
  if (d->smoother == HMG_SMOOTH_BLOCKJACOBI) {
    if (d->smooth_prec != HMG_PREC_FP64) { set_error("block Jacobi smoothing runs in FP64 only"); return HMG_EINVAL; }
    long long mi = 1;
    for (int a = 0; a < d->dim; ++a) mi *= d->order - 1;
    if (mi > kMaxBlock) {
      set_error("block Jacobi: (p-1)^d = " + std::to_string(mi) + " interior nodes per element exceeds " +
                std::to_string(kMaxBlock));
      return HMG_EINVAL;
    }
  }
  if (d->nu_pre < 0 || d->nu_post < 0 || d->nu_pre > 64 || d->nu_post > 64) { set_error("bad nu"); return HMG_EINVAL; }
  if (!(fabs(d->warp_amp) * M_PI < 1.0)) { set_error("|warp_amp| * pi must be < 1"); return HMG_EINVAL; }
  if (!(d->mu_a > 0.0) || !(d->mu_a + (d->mu_b < 0 ? d->mu_b * d->dim : 0.0) > 0.0)) {
    set_error("mu must stay positive"); return HMG_EINVAL;
  }
  if (d->smoother == HMG_SMOOTH_CHEB && (d->arnoldi_iters < 1 || !(d->cheb_lo_frac > 0.0 && d->cheb_lo_frac < 1.0) ||
                                         !(d->cheb_safety > 0.0))) {
    set_error("bad Chebyshev parameters"); return HMG_EINVAL;
  }
  if (d->smooth_prec < HMG_PREC_FP64 || d->smooth_prec > HMG_PREC_BF16) { set_error("bad smooth_prec"); return HMG_EINVAL; }
  if (d->fp64_arith != HMG_ARITH_FP64 && d->fp64_arith != HMG_ARITH_DF64) { set_error("bad fp64_arith"); return HMG_EINVAL; }
  return HMG_OK;
}

// ---- 1D transfer stencils (Sec. 2.2: P_ij = coarse basis j at fine node i, per axis) ----
hmg_status build_axis(ProblemImpl& P, const Level& f, const Level& c, int a, Axis1D* Pax, Axis1D* PTax) {
  const int ratio = f.m.E[a] / c.m.E[a];
  if (ratio != 1 && ratio != 2) { set_error("levels not nested"); return HMG_EINVAL; }
  const int nf = (int)f.m.Nn[a], ncn = (int)c.m.Nn[a];
  const int pf = f.m.p, pc = c.m.p;
  std::vector<std::vector<std::pair<int, double>>> rows(nf), cols(ncn);
  double vals[kMaxN];
  for (int I = 0; I < nf; ++I) {
    const int ef = std::min(I / pf, f.m.E[a] - 1);
    const int i = I - ef * pf;
    const int ec = ef / ratio;
    const double xi = ((ef % ratio) + f.basis.r[i]) / ratio;
    lagrange_row(c.basis.r, pc + 1, xi, vals);
    for (int k = 0; k <= pc; ++k) {
      if (vals[k] == 0.0) continue;
      const int J = ec * pc + k;
      rows[I].push_back({J, vals[k]});
      cols[J].push_back({I, vals[k]});
    }
  }
  auto upload = [&](const std::vector<std::vector<std::pair<int, double>>>& R, int n_in, Axis1D* out) -> hmg_status {
    std::vector<int> rp(1, 0), ci;
    std::vector<double> v;
    std::vector<float> v32;
    for (auto& row : R) {
      for (auto& e : row) { ci.push_back(e.first); v.push_back(e.second); v32.push_back((float)e.second); }
      rp.push_back((int)ci.size());
    }
    out->n_out = (int)R.size();
    out->n_in = n_in;
    TRY(P.alloc((void**)&out->rowptr, rp.size() * sizeof(int)));
    TRY(P.alloc((void**)&out->col, ci.size() * sizeof(int)));
    TRY(P.alloc((void**)&out->val, v.size() * sizeof(double)));
    TRY(P.alloc((void**)&out->val32, v32.size() * sizeof(float)));
    // pageable sources: each asynchronous copy has staged them when it returns
    cudaStream_t s = P.setup_stream;
    TRY(cudaMemcpyAsync(out->rowptr, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyAsync(out->col, ci.data(), ci.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyAsync(out->val, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyAsync(out->val32, v32.data(), v32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    return HMG_OK;
  };
  CHECK(upload(rows, ncn, Pax));
  CHECK(upload(cols, nf, PTax));
  return HMG_OK;
}

// ---- precision-generic accessors ----
template <typename T> struct Acc;
template <> struct Acc<double> {
  static double* b(Level& l) { return l.b; }
  static double* x(Level& l) { return l.x; }
  static double* r(Level& l) { return l.r; }
  static double* d(Level& l) { return l.d; }
  static const double* dinv(Level& l) { return l.dinv; }
  static void* scratch(void* p) { return p; }
};
template <> struct Acc<float> {
  static float* b(Level& l) { return l.b32; }
  static float* x(Level& l) { return l.x32; }
  static float* r(Level& l) { return l.r32; }
  static float* d(Level& l) { return l.d32; }
  static const float* dinv(Level& l) { return l.dinv32; }
};

hmg_status apply_level(ProblemImpl& P, int k, const double* x, double* y, double alpha, cudaStream_t s) {
  Level& l = P.L[k];
  if (k == 0 && !P.capturing) P.fine_applies++;
  TRY(launch_apply_f64(l.m, l.basis, x, y, l.G, alpha, P.err, s, l.v64, l.Ke, l.Gdf));
  return HMG_OK;
}
hmg_status apply_level(ProblemImpl& P, int k, const float* x, float* y, float alpha, cudaStream_t s) {
  Level& l = P.L[k];
  if (k == 0 && !P.capturing) P.fine_applies++;
  TRY(launch_apply_low(l.m, l.basis, x, y, l.Glow, l.gsc, alpha, P.desc.smooth_prec, s, l.v32, &l.tc, P.err));
  return HMG_OK;
}

// x_f (=, or += if acc) P x_c between level k (fine) and k+1 (coarse).
template <typename T>
hmg_status prolong(ProblemImpl& P, int k, const T* xc, T* xf, bool acc, cudaStream_t s) {
  Level& f = P.L[k];
  Level& c = P.L[k + 1];
  const int dim = f.m.dim;
  long long od[3] = {c.m.Nn[0], c.m.Nn[1], c.m.Nn[2]};
  const T* in = xc;
  T* bufs[2] = {(T*)P.t1, (T*)P.t2};
  for (int a = 0; a < dim; ++a) {
    od[a] = f.m.Nn[a];
    const bool last = (a == dim - 1);
    T* out = last ? xf : bufs[a & 1];
    TRY(axis_pass<T>(in, out, od, a, f.P[a], a == 0, last, last && acc, s));
    in = out;
  }
  return HMG_OK;
}

// r_c = P^T r_f between level k (fine) and k+1 (coarse).
template <typename T>
hmg_status restrict_(ProblemImpl& P, int k, const T* rf, T* rc, cudaStream_t s) {
  Level& f = P.L[k];
  Level& c = P.L[k + 1];
  const int dim = f.m.dim;
  long long od[3] = {f.m.Nn[0], f.m.Nn[1], f.m.Nn[2]};
  const T* in = rf;
  T* bufs[2] = {(T*)P.t1, (T*)P.t2};
  for (int a = 0; a < dim; ++a) {
    od[a] = c.m.Nn[a];
    const bool last = (a == dim - 1);
    T* out = last ? rc : bufs[a & 1];
    TRY(axis_pass<T>(in, out, od, a, f.PT[a], a == 0, last, 0, s));
    in = out;
  }
  return HMG_OK;
}

// `steps` smoothing steps on level k. zero: x is taken as 0 on input. Each step's residual
// r = b - A x is formed by the apply into r holding b; the update kernel of one step writes
// r = b for the next step (no separate copy). With leave_r_b, r = b on return.
template <typename T>
hmg_status smooth(ProblemImpl& P, int k, const T* b, T* x, int steps, bool zero, cudaStream_t s,
                  bool leave_r_b = false) {
  Level& l = P.L[k];
  const hmg_desc& D = P.desc;
  const long long n = l.m.N;
  T* r = Acc<T>::r(l);
  T* d = Acc<T>::d(l);
  const T* dinv = Acc<T>::dinv(l);
  if (steps <= 0) {
    if (zero) TRY(cudaMemsetAsync(x, 0, n * sizeof(T), s));
    if (leave_r_b) TRY(cudaMemcpyAsync(r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return HMG_OK;
  }
  bool r_is_b = false;
  auto residual = [&]() -> hmg_status {
    if (!r_is_b) TRY(cudaMemcpyAsync(r, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return apply_level(P, k, x, r, (T)-1, s);
  };
  if (D.smoother == HMG_SMOOTH_JACOBI || D.smoother == HMG_SMOOTH_L1JACOBI) {  // same step, other D
    const T w = (T)D.omega;
    for (int st = 0; st < steps; ++st) {
      const bool reset = st + 1 < steps || leave_r_b;
      if (st == 0 && zero) {
        TRY(jacobi_first<T>(x, b, dinv, n, w, s, reset ? r : nullptr));
      } else {
        CHECK(residual());
        TRY(jacobi_step<T>(x, r, b, dinv, n, w, reset ? 1 : 0, s));
      }
      r_is_b = reset;
    }
    return HMG_OK;
  }
  if (D.smoother == HMG_SMOOTH_BLOCKJACOBI) {
    if constexpr (std::is_same<T, double>::value) {
      // element-interior blocks (inverses in Kb) and the diagonal on shared nodes touch disjoint
      // unknowns; the block part reads r before the point step resets it to b
      const double w = D.omega;
      const double* ds = l.Kb ? l.dinv_s : l.dinv;
      for (int st = 0; st < steps; ++st) {
        const bool reset = st + 1 < steps || leave_r_b;
        if (st == 0 && zero) {
          TRY(jacobi_first<double>(x, b, ds, n, w, s, reset ? r : nullptr));
          if (l.Kb) TRY(launch_block_smooth(l.m, l.Kb, b, x, w, s));
        } else {
          CHECK(residual());
          if (l.Kb) TRY(launch_block_smooth(l.m, l.Kb, r, x, w, s));
          TRY(jacobi_step<double>(x, r, b, ds, n, w, reset ? 1 : 0, s));
        }
        r_is_b = reset;
      }
      return HMG_OK;
    } else {
      set_error("block Jacobi smoothing runs in FP64 only");
      return HMG_EINVAL;
    }
  }
  // Chebyshev acceleration of Jacobi on [lo, hi] (Saad, Iterative Methods, Alg. 12.1)
  const double hi = D.cheb_safety * l.lam, lo = D.cheb_lo_frac * hi;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int st = 0; st < steps; ++st) {
    const bool reset = st + 1 < steps || leave_r_b;
    if (st == 0) {
      if (zero) {
        TRY(cheb_first<T>(x, d, b, dinv, n, (T)(1.0 / theta), s, reset ? r : nullptr));
      } else {
        CHECK(residual());
        TRY(cheb_step<T>(x, d, r, b, dinv, n, (T)0, (T)(1.0 / theta), reset ? 1 : 0, s));
      }
    } else {
      CHECK(residual());
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      TRY(cheb_step<T>(x, d, r, b, dinv, n, (T)(rho_new * rho), (T)(2.0 * rho_new / delta), reset ? 1 : 0, s));
      rho = rho_new;
    }
    r_is_b = reset;
  }
  return HMG_OK;
}

hmg_status coarse(ProblemImpl& P, int k, const double* b, double* x, cudaStream_t s) {
  Level& l = P.L[k];
  TRY(cudaMemsetAsync(x, 0, l.m.N * sizeof(double), s));
  if (l.nI > 0) TRY(coarse_solve(l.Ainv, b, x, l.gmap, l.nI, s));
  return HMG_OK;
}
hmg_status coarse(ProblemImpl& P, int k, const float* b, float* x, cudaStream_t s) {
  Level& l = P.L[k];
  TRY(cudaMemsetAsync(x, 0, l.m.N * sizeof(float), s));
  if (l.nI > 0) TRY(coarse_solve_f32(l.Ainv, b, x, l.gmap, l.nI, s));
  return HMG_OK;
}

// One V(nu_pre, nu_post) cycle on level k for A_k x = b (zero: x starts at 0).
template <typename T>
hmg_status vcycle(ProblemImpl& P, int k, const T* b, T* x, bool zero, cudaStream_t s) {
  const int last = (int)P.L.size() - 1;
  if (k == last) return coarse(P, k, b, x, s);
  Level& l = P.L[k];
  Level& c = P.L[k + 1];
  const long long n = l.m.N;
  T* r = Acc<T>::r(l);
  CHECK(smooth<T>(P, k, b, x, P.desc.nu_pre, zero, s, true));  // leaves r = b
  CHECK(apply_level(P, k, x, r, (T)-1, s));
  CHECK(restrict_<T>(P, k, r, Acc<T>::b(c), s));
  CHECK(vcycle<T>(P, k + 1, Acc<T>::b(c), Acc<T>::x(c), true, s));
  CHECK(prolong<T>(P, k, Acc<T>::x(c), x, true, s));
  CHECK(smooth<T>(P, k, b, x, P.desc.nu_post, false, s));
  return HMG_OK;
}

// z = B r on the finest level (FP64 in and out; FP32 internally for the mixed form).
hmg_status precondition(ProblemImpl& P, const double* r, double* z, cudaStream_t s) {
  if (P.desc.smooth_prec != HMG_PREC_FP64 && P.L.size() > 1) {
    Level& l = P.L[0];
    TRY(to_f32(l.b32, r, l.m.N, s));
    CHECK(vcycle<float>(P, 0, l.b32, l.x32, true, s));
    TRY(to_f64(z, l.x32, l.m.N, s));
    return HMG_OK;
  }
  return vcycle<double>(P, 0, r, z, true, s);
}

hmg_status dot_to(ProblemImpl& P, const double* x, const double* y, long long n, int op, int idx, int aux,
                  bool to_host, cudaStream_t s) {
  TRY(dot_partial(x, y, n, P.partial, s));
  TRY(finish(P.partial, n, P.S, op, idx, aux, to_host ? P.hostS : nullptr, s));
  return HMG_OK;
}

// New rho = (z, r) and beta of PCG (Algorithm 1). With a 16-bit V-cycle the preconditioner is
// only nearly linear, so beta takes the flexible (Polak-Ribiere) form
// (z_new, r_new - r_old) / (z_old, r_old) = -(z_new, A p_old) / (p_old, A p_old), using h = A p
// still held in P.ph; otherwise the standard (z_new, r_new) / (z_old, r_old).
hmg_status pcg_rho_beta(ProblemImpl& P, const double* z, const double* r, long long n, cudaStream_t s) {
  if (P.desc.smooth_prec == HMG_PREC_FP16 || P.desc.smooth_prec == HMG_PREC_BF16) {
    CHECK(dot_to(P, z, P.ph, n, FIN_NEG_RATIO, S_BETA, S_PH, false, s));
    return dot_to(P, z, r, n, FIN_STORE, S_RHO, 0, false, s);
  }
  return dot_to(P, z, r, n, FIN_RHO_BETA, S_RHO, S_BETA, false, s);
}

// lambda_max of D^-1 A_k by m Arnoldi steps (Sec. 3.2.2). The orthogonalization is classical
// Gram-Schmidt applied twice (CGS2: one fused multi-dot, one fused multi-axpy per pass), which
// gives the Hessenberg matrix of modified Gram-Schmidt up to rounding with 6 launches per step
// instead of 3 (j+1).
hmg_status arnoldi(ProblemImpl& P, int k, cudaStream_t s) {
  Level& l = P.L[k];
  const int m = (int)std::min<long long>(P.desc.arnoldi_iters, l.nI);
  if (m < 1) { l.lam = 1.0; return HMG_OK; }
  const long long n = l.m.N;
  double *Vb = nullptr, *Hd = nullptr, *part = nullptr, *coef = nullptr;
  std::vector<void*> tmp;
  auto cleanup = [&]() { for (void* p : tmp) dev_free(p, s); };
  auto get = [&](double** ptr, size_t count) -> bool {
    if (dev_alloc((void**)ptr, count * sizeof(double), s) != cudaSuccess) return false;
    tmp.push_back(*ptr);
    return true;
  };
  if (!get(&Vb, (size_t)(m + 1) * n) || !get(&Hd, (size_t)(m + 1) * m) ||
      !get(&part, (size_t)(m + 1) * red_blocks(n)) || !get(&coef, (size_t)(m + 1))) {
    cleanup();
    set_error("arnoldi alloc");
    return HMG_ENOMEM;
  }
  auto V = [&](int j) { return Vb + (long long)j * n; };
  hmg_status st = [&]() -> hmg_status {
    TRY(cudaMemsetAsync(Hd, 0, (m + 1) * m * sizeof(double), s));
    const unsigned long long seed = (P.desc.arnoldi_seed ? P.desc.arnoldi_seed : 0x1402593800000000ull) + (unsigned long long)k;
    TRY(start_vector(V(0), l.m, seed, s));
    TRY(dot_partial(V(0), V(0), n, P.partial, s));
    TRY(finish(P.partial, n, P.S, FIN_SQRT, S_TMP, 0, nullptr, s));
    TRY(div_dev(V(0), V(0), n, P.S + S_TMP, s));
    for (int j = 0; j < m; ++j) {
      double* w = V(j + 1);
      TRY(cudaMemsetAsync(w, 0, n * sizeof(double), s));
      TRY(launch_apply_f64(l.m, l.basis, V(j), w, l.G, 1.0, P.err, s, l.v64, l.Ke, l.Gdf));
      TRY(scale_by(w, l.dinv, n, s));
      for (int pass = 0; pass < 2; ++pass)  // H[0..j][j] accumulates both passes
        TRY(project_out(w, Vb, n, j + 1, n, part, coef, Hd + j, m, s));
      TRY(dot_partial(w, w, n, P.partial, s));
      TRY(finish(P.partial, n, Hd, FIN_SQRT, (j + 1) * m + j, 0, nullptr, s));
      if (j + 1 < m) TRY(div_dev(w, w, n, Hd + (j + 1) * m + j, s));
    }
    std::vector<double> H((m + 1) * m);
    TRY(cudaMemcpyAsync(H.data(), Hd, H.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    l.lam = hessenberg_max_real_eig(H.data(), m);
    if (!(l.lam > 0.0) || !isfinite(l.lam)) { set_error("Chebyshev bound estimate failed"); return HMG_ENAN; }
    return HMG_OK;
  }();
  cleanup();
  return st;
}

// ---- autotuning of the apply block shape -------------------------------------------------
// For each level, time the kernel variants (block shapes, and for FP64 TMA staging) with CUDA events on the
// level's own buffers and keep the fastest; results are cached per (device, dim, order, element
// count, precision) for the process. HMG_AUTOTUNE=0 in the environment keeps variant 0.
constexpr long long kTuneMinPoints = 32768;  // Gauss points below which a level is not tuned

bool autotune_on() {
  static const bool on = [] {
    const char* v = getenv("HMG_AUTOTUNE");
    return !(v && v[0] == '0');
  }();
  return on;
}

// Autotuner decisions, keyed by (device, dim, order, elements, precision kind), and the first
// decision of each size class under elements = -k (element counts in [2^(k-1), 2^k)), which a level
// without its own entry reuses. With HMG_AUTOTUNE_CACHE=<file> they persist across processes: the
// file's lines "device dim order elements kind variant" are read once, and new decisions are
// appended, so a later process (for instance one run under a profiler, whose timings would be
// distorted) reuses them instead of timing again.
using TuneKey = std::tuple<int, int, int, long long, int>;
std::map<TuneKey, int>& tune_cache() {
  static std::map<TuneKey, int> cache = [] {
    std::map<TuneKey, int> m;
    if (const char* f = getenv("HMG_AUTOTUNE_CACHE")) {
      if (FILE* fp = fopen(f, "r")) {
        int dev, dim, p, kind, v;
        long long ne;
        while (fscanf(fp, "%d %d %d %lld %d %d", &dev, &dim, &p, &ne, &kind, &v) == 6)
          m[std::make_tuple(dev, dim, p, ne, kind)] = v;
        fclose(fp);
      }
    }
    return m;
  }();
  return cache;
}

void tune_cache_store(const TuneKey& k, int v) {
  tune_cache()[k] = v;
  if (const char* f = getenv("HMG_AUTOTUNE_CACHE")) {
    if (FILE* fp = fopen(f, "a")) {
      fprintf(fp, "%d %d %d %lld %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
              std::get<4>(k), v);
      fclose(fp);
    }
  }
}

// Apply variants a level can run: FP64 (the point-parallel shapes, stored element matrices, the
// FP64 pencil form) or the mixed V-cycle's operator (pencil factor-load timings, tensor-core form).
std::vector<int> level_variants(const Level& l, bool vcycle_op) {
  if (!vcycle_op) return apply64_variants(l.m.dim, l.m.p + 1, l.Ke != nullptr);
  std::vector<int> v;
  for (int k = 0; k < kApplyLowVariants; ++k) v.push_back(k);
  if (l.tc.G) v.push_back(kApplyLowTc);
  return v;
}

hmg_status tune_level(ProblemImpl& P, Level& l, cudaStream_t s) {
  if (!autotune_on()) return HMG_OK;
  // tiny levels run at the launch-latency floor whatever the block shape: variant 0 unless the
  // decision cache names one
  const bool tiny = l.m.nelem * np_of(l.m) < kTuneMinPoints;
  static std::mutex mu;
  std::map<TuneKey, int>& cache = [&]() -> std::map<TuneKey, int>& {
    std::lock_guard<std::mutex> lk(mu);
    return tune_cache();
  }();
  int dev = 0;
  TRY(cudaGetDevice(&dev));
  const bool mixed = l.Glow != nullptr;
  for (int prec = 0; prec < (mixed ? 2 : 1); ++prec) {
    const int kind = prec == 0 ? 0 : P.desc.smooth_prec;
    const auto key = std::make_tuple(dev, l.m.dim, l.m.p, l.m.nelem, kind);
    // size class: element counts in [2^(k-1), 2^k) share a decision (entry -k), so a stream of
    // similar problems (a server's) times each class once
    int cls = 0;
    for (long long n = l.m.nelem; n > 0; n >>= 1) ++cls;
    const auto ckey = std::make_tuple(dev, l.m.dim, l.m.p, -(long long)cls, kind);
    {
      std::lock_guard<std::mutex> lk(mu);
      const std::vector<int> cand = level_variants(l, prec != 0);
      auto runnable = [&](std::map<TuneKey, int>::iterator it) {
        return it != cache.end() && std::find(cand.begin(), cand.end(), it->second) != cand.end();
      };
      auto it = cache.find(key);
      if (!runnable(it)) it = cache.find(ckey);
      if (runnable(it)) {  // a decision this level can run: its own, else its size class's
        (prec ? l.v32 : l.v64) = it->second;
        continue;
      }
    }
    if (tiny) continue;
    cudaEvent_t e0, e1;
    TRY(cudaEventCreate(&e0));
    TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int bv = 0;
    cudaError_t err = cudaSuccess;
    for (int v : level_variants(l, prec != 0)) {
      if (err != cudaSuccess) break;
      auto run = [&]() {
        if (prec == 0) return launch_apply_f64(l.m, l.basis, l.x, l.r, l.G, 1.0, P.err, s, v, l.Ke);
        return launch_apply_low(l.m, l.basis, l.x32, l.r32, l.Glow, l.gsc, 1.0f, P.desc.smooth_prec, s, v, &l.tc,
                                P.err);
      };
      // warm-up (also opts the kernel into its smem); a variant this level cannot launch (its
      // configuration refused, no fault) is skipped
      if ((err = run()) != cudaSuccess) {
        if (err == cudaErrorInvalidValue || err == cudaErrorInvalidConfiguration ||
            err == cudaErrorLaunchOutOfResources) {
          cudaGetLastError();
          err = cudaSuccess;
          continue;
        }
        break;
      }
      if ((err = cudaEventRecord(e0, s)) != cudaSuccess) break;
      for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = run();
      if (err == cudaSuccess) err = cudaEventRecord(e1, s);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err == cudaSuccess && Phase::timing())
        fprintf(stderr, "hmg autotune timing: dim %d p %d elements %lld %s variant %d: %.4f ms per apply\n", l.m.dim,
                l.m.p, l.m.nelem, kind == 0 ? "fp64" : (kind == HMG_PREC_FP32 ? "fp32" : "16-bit"), v, ms / 3);
      if (err == cudaSuccess && ms < best) {
        best = ms;
        bv = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(err);
    (prec ? l.v32 : l.v64) = bv;
    if (Phase::timing())
      fprintf(stderr, "hmg autotune: dim %d p %d elements %lld %s -> variant %d (%.4f ms per apply)\n", l.m.dim,
              l.m.p, l.m.nelem, kind == 0 ? "fp64" : (kind == HMG_PREC_FP32 ? "fp32" : "16-bit"), bv, best / 3);
    std::lock_guard<std::mutex> lk(mu);
    tune_cache_store(key, bv);
    if (cache.find(ckey) == cache.end()) tune_cache_store(ckey, bv);
  }
  TRY(cudaMemsetAsync(l.r, 0, l.m.N * sizeof(double), s));
  if (mixed) TRY(cudaMemsetAsync(l.r32, 0, l.m.N * sizeof(float), s));
  return HMG_OK;
}

// Largest coarsest level for the dense exact inverse: the paper's order-16 h-hierarchy on a 32^2
// mesh ends on 127^2 = 16,129 unknowns (a 2.1 GB matrix, ~4e12 flops of Gauss-Jordan at setup).
constexpr long long kMaxCoarse = 20000;

hmg_status build_coarse(ProblemImpl& P, Level& l, cudaStream_t s) {
  const long long nI = l.nI;
  if (nI == 0) return HMG_OK;
  if (nI > kMaxCoarse) {
    set_error("coarsest level has " + std::to_string(nI) + " unknowns; the dense exact solve allows " + std::to_string(kMaxCoarse) + ": add levels");
    return HMG_EINVAL;
  }
  TRY(P.alloc((void**)&l.Ainv, (size_t)nI * nI * sizeof(double)));
  std::vector<long long> gm;
  gm.reserve(nI);
  for (long long g = 0; g < l.m.N; ++g) {
    const long long I = g % l.m.Nn[0], r = g / l.m.Nn[0], J = r % l.m.Nn[1], K = r / l.m.Nn[1];
    bool bd = I == 0 || I == l.m.Nn[0] - 1 || J == 0 || J == l.m.Nn[1] - 1;
    if (l.m.dim == 3) bd = bd || K == 0 || K == l.m.Nn[2] - 1;
    if (!bd) gm.push_back(g);
  }
  TRY(P.alloc((void**)&l.gmap, nI * sizeof(long long)));
  TRY(cudaMemcpyAsync(l.gmap, gm.data(), nI * sizeof(long long), cudaMemcpyHostToDevice, s));
  TRY(launch_elem_dense(l.m, l.basis, l.G, l.Ainv, nI, s));
  double* work = nullptr;
  int* bad = nullptr;
  TRY(dev_alloc((void**)&work, blocked_gj_work_doubles(nI) * sizeof(double), s));
  if (dev_alloc((void**)&bad, sizeof(int), s) != cudaSuccess) { dev_free(work, s); set_error("alloc"); return HMG_ENOMEM; }
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) e = blocked_gauss_jordan_inverse(l.Ainv, nI, work, bad, s);
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  dev_free(work, s);
  dev_free(bad, s);
  TRY(e);
  TRY(e2);
  if (hbad) { set_error("coarsest operator: a non-positive pivot (not positive definite)"); return HMG_EINVAL; }
  return HMG_OK;
}

hmg_status setup_impl(ProblemImpl& P, cudaStream_t s) {
  const hmg_desc& D = P.desc;
  P.setup_stream = s;
  TRY(cudaStreamCreateWithFlags(&P.own, cudaStreamNonBlocking));
  std::vector<std::pair<std::vector<int>, int>> shapes;
  CHECK(level_shapes(D, shapes));
  P.L.resize(shapes.size());
  size_t max_stage = 0, max_tbuf = 0;
  for (size_t k = 0; k < shapes.size(); ++k) {
    Level& l = P.L[k];
    l.m = make_mesh(D.dim, shapes[k].first.data(), shapes[k].second);
    make_basis(l.m.p, &l.basis);
    l.nI = interior_count(l.m);
    max_stage = std::max(max_stage, (size_t)(l.m.nelem * np_of(l.m) * D.dim * (D.dim + 1)) * sizeof(double));
  }
  // transfer intermediates: largest partial product over all passes
  for (size_t k = 0; k + 1 < P.L.size(); ++k) {
    const Mesh& f = P.L[k].m;
    const Mesh& c = P.L[k + 1].m;
    long long od[3] = {c.Nn[0], c.Nn[1], c.Nn[2]};
    for (int a = 0; a < D.dim; ++a) { od[a] = f.Nn[a]; max_tbuf = std::max(max_tbuf, (size_t)(od[0] * od[1] * od[2])); }
    long long rd[3] = {f.Nn[0], f.Nn[1], f.Nn[2]};
    for (int a = 0; a < D.dim; ++a) { rd[a] = c.Nn[a]; max_tbuf = std::max(max_tbuf, (size_t)(rd[0] * rd[1] * rd[2])); }
  }
  Phase ph_all("setup", s);
  TRY(P.alloc((void**)&P.S, 64 * sizeof(double)));
  TRY(P.alloc((void**)&P.err, sizeof(int)));
  TRY(P.alloc((void**)&P.partial, kRedBlocks * sizeof(double)));
  P.hostS = static_cast<double*>(pinned_alloc(16 * sizeof(double)));
  if (!P.hostS) { set_error("pinned host allocation failed"); return HMG_ENOMEM; }
  TRY(P.alloc(&P.t1, max_tbuf * sizeof(double)));
  TRY(P.alloc(&P.t2, max_tbuf * sizeof(double)));
  const long long N0 = P.L[0].m.N;
  TRY(P.alloc((void**)&P.pr, N0 * sizeof(double)));
  TRY(P.alloc((void**)&P.pz, N0 * sizeof(double)));
  TRY(P.alloc((void**)&P.pp, N0 * sizeof(double)));
  TRY(P.alloc((void**)&P.ph, N0 * sizeof(double)));
  TRY(P.alloc((void**)&P.gb, N0 * sizeof(double)));
  TRY(P.alloc((void**)&P.gu, N0 * sizeof(double)));
  TRY(P.alloc((void**)&P.ctrl, 4 * sizeof(int)));
  P.host_ctrl = static_cast<int*>(pinned_alloc(4 * sizeof(int)));
  if (!P.host_ctrl) { set_error("pinned host allocation failed"); return HMG_ENOMEM; }

  double* Jstage = nullptr;
  int* bad = nullptr;
  TRY(dev_alloc((void**)&Jstage, max_stage, s));
  if (dev_alloc((void**)&bad, sizeof(int), s) != cudaSuccess) { dev_free(Jstage, s); set_error("alloc"); return HMG_ENOMEM; }
  // user geometry / coefficient: finest coordinates, a coarse level's coordinates, Gauss points, mu
  std::vector<void*> tmp;
  auto talloc = [&](void** ptr, size_t bytes) -> hmg_status {
    if (dev_alloc(ptr, bytes, s) != cudaSuccess) { set_error("device allocation failed"); return HMG_ENOMEM; }
    tmp.push_back(*ptr);
    return HMG_OK;
  };
  double *X0 = nullptr, *Xk = nullptr, *xq_d = nullptr, *mu_d = nullptr;
  std::vector<double> xq_h, mu_h;
  hmg_status st = [&]() -> hmg_status {
    const long long nq0 = P.L[0].m.nelem * np_of(P.L[0].m);
    if (D.node_xyz) {
      TRY(P.alloc((void**)&X0, (size_t)D.dim * N0 * sizeof(double)));  // kept: hmg_node_coords
      P.X0 = X0;
      CHECK(talloc((void**)&Xk, (size_t)D.dim * N0 * sizeof(double)));
      TRY(cudaMemcpyAsync(X0, D.node_xyz, (size_t)D.dim * N0 * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    if (D.mu_fn) {
      CHECK(talloc((void**)&xq_d, (size_t)D.dim * nq0 * sizeof(double)));
      CHECK(talloc((void**)&mu_d, (size_t)nq0 * sizeof(double)));
    }
    const bool mixed = D.smooth_prec != HMG_PREC_FP64;
    for (size_t k = 0; k < P.L.size(); ++k) {
      Phase ph("setup: level geometry, diagonal", s);
      Level& l = P.L[k];
      const long long n = l.m.N;
      const long long gsz = l.m.nelem * np_of(l.m);
      TRY(P.alloc((void**)&l.G, gsz * nc_of(D.dim) * sizeof(double) + 256));  // TMA tail padding
      TRY(P.alloc((void**)&l.wdetJ, gsz * sizeof(double)));
      TRY(P.alloc((void**)&l.dinv, n * sizeof(double)));
      TRY(P.alloc((void**)&l.b, n * sizeof(double)));
      TRY(P.alloc((void**)&l.x, n * sizeof(double)));
      TRY(P.alloc((void**)&l.r, n * sizeof(double)));
      TRY(P.alloc((void**)&l.d, n * sizeof(double)));
      TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
      const double* coords = nullptr;
      if (D.node_xyz) {
        if (k > 0) TRY(launch_level_coords(P.L[0].m, P.L[0].basis, X0, l.m, l.basis, Xk, s));
        coords = k == 0 ? X0 : Xk;
      }
      TRY(launch_geom_stage(l.m, l.basis, D.warp_amp, coords, Jstage, s));
      const double* mu_arr = nullptr;
      if (D.mu_fn) {  // the user's coefficient at this level's Gauss points
        const size_t nq = (size_t)gsz;
        xq_h.resize((size_t)D.dim * nq);
        mu_h.assign(nq, 0.0);
        TRY(launch_extract_xq(l.m, l.basis, Jstage, xq_d, s));
        TRY(cudaMemcpyAsync(xq_h.data(), xq_d, xq_h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        TRY(cudaStreamSynchronize(s));
        D.mu_fn(nq, xq_h.data(), mu_h.data(), D.mu_user);
        for (double v : mu_h)
          if (!(v > 0.0) || !std::isfinite(v)) { set_error("mu_fn returned a non-positive or non-finite value"); return HMG_EINVAL; }
        TRY(cudaMemcpyAsync(mu_d, mu_h.data(), nq * sizeof(double), cudaMemcpyHostToDevice, s));
        mu_arr = mu_d;
      }
      TRY(launch_geom_point(l.m, l.basis, D.mu_a, D.mu_b, D.mu_k, mu_arr, Jstage, l.G, l.wdetJ, bad, s));
      int hbad = 0;
      TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      TRY(cudaStreamSynchronize(s));
      if (hbad) { set_error("non-positive Jacobian determinant: the mapped mesh is folded"); return HMG_EINVAL; }
      // diagonal -> D^-1 (the diagonal is accumulated in l.r, then cleared)
      TRY(launch_diag(l.m, l.basis, l.G, l.r, s));
      // low orders, FP64 applies of a V-cycle level (all levels in FP64; the finest otherwise):
      // element matrices for the dense-apply variant, which the autotuner may pick
      if (l.m.p + 1 <= kMaxNDense && k + 1 < P.L.size() && (k == 0 || D.smooth_prec == HMG_PREC_FP64)) {
        const long long np = np_of(l.m);
        TRY(P.alloc((void**)&l.Ke, (size_t)l.m.nelem * np * np * sizeof(double)));
        TRY(launch_elem_mats(l.m, l.basis, l.G, l.Ke, s));
      }
      if (D.smoother == HMG_SMOOTH_L1JACOBI && k + 1 < P.L.size()) {
        // l1 row norms sum_j |a_ij|: along an axis a row couples at most 2p+1 consecutive nodes,
        // so the nodes of one color class (indices mod 2p+1) meet each row at most once, and
        // y = A (indicator of the class) holds one entry a_ij per row
        TRY(cudaMemsetAsync(l.r, 0, n * sizeof(double), s));
        const int period = 2 * l.m.p + 1;
        int pc[3] = {1, 1, 1};
        for (int a = 0; a < D.dim; ++a) pc[a] = (int)std::min<long long>(period, l.m.Nn[a]);
        for (int c2 = 0; c2 < pc[2]; ++c2)
          for (int c1 = 0; c1 < pc[1]; ++c1)
            for (int c0 = 0; c0 < pc[0]; ++c0) {
              TRY(color_indicator(l.x, l.m, period, c0, c1, c2, s));
              TRY(cudaMemsetAsync(l.d, 0, n * sizeof(double), s));
              TRY(launch_apply_f64(l.m, l.basis, l.x, l.d, l.G, 1.0, P.err, s, 0));
              TRY(accum_abs(l.r, l.d, n, s));
            }
        TRY(cudaMemsetAsync(l.x, 0, n * sizeof(double), s));
        TRY(cudaMemsetAsync(l.d, 0, n * sizeof(double), s));
      }
      TRY(dinv_from_diag(l.r, l.dinv, n, s));
      TRY(cudaMemsetAsync(l.r, 0, n * sizeof(double), s));
      if (D.smoother == HMG_SMOOTH_BLOCKJACOBI && k + 1 < P.L.size() && block_size_of(l.m) > 0) {
        // element-interior blocks of K_e, inverted in place; D^-1 kept on the shared nodes only
        const int MI = block_size_of(l.m);
        double* Kw = nullptr;  // blocks and their in-place inversion (setup temporary)
        CHECK(talloc((void**)&Kw, (size_t)l.m.nelem * MI * MI * sizeof(double)));
        TRY(P.alloc((void**)&l.Kb, (size_t)packed_block_doubles(l.m.nelem, MI) * sizeof(double)));
        TRY(P.alloc((void**)&l.dinv_s, n * sizeof(double)));
        TRY(launch_elem_blocks(l.m, l.basis, l.G, Kw, s));
        TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        TRY(launch_block_invert(Kw, l.m.nelem, MI, bad, s));
        TRY(launch_block_pack(Kw, l.Kb, l.m.nelem, MI, s));
        TRY(cudaMemcpyAsync(l.dinv_s, l.dinv, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        TRY(launch_mask_elem_interior(l.dinv_s, l.m, s));
        int hb = 0;
        TRY(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        TRY(cudaStreamSynchronize(s));
        tmp.erase(std::find(tmp.begin(), tmp.end(), (void*)Kw));
        dev_free(Kw, s);
        if (hb) { set_error("block Jacobi: an element-interior block is not positive definite"); return HMG_EINVAL; }
      }
      if (mixed) {
        TRY(P.alloc((void**)&l.Glow, low_factor_bytes(l.m, D.smooth_prec) + 256));  // prefetch rounding
        if (D.smooth_prec != HMG_PREC_FP32) TRY(P.alloc((void**)&l.gsc, l.m.nelem * sizeof(float)));
        if (tc16_supported(l.m, D.smooth_prec)) {  // tensor-core form: its factor layout and Phi image
          std::vector<unsigned char> img;
          tc16_phi_image(l.basis, img, &l.tc.vsc);
          void *phi = nullptr, *gtc = nullptr;
          TRY(P.alloc(&phi, img.size()));
          TRY(cudaMemcpyAsync(phi, img.data(), img.size(), cudaMemcpyHostToDevice, s));
          TRY(P.alloc(&gtc, tc16_factor_bytes(l.m)));
          l.tc.phi = phi;
          l.tc.G = gtc;
        }
        TRY(P.alloc((void**)&l.dinv32, n * sizeof(float)));
        TRY(P.alloc((void**)&l.b32, n * sizeof(float)));
        TRY(P.alloc((void**)&l.x32, n * sizeof(float)));
        TRY(P.alloc((void**)&l.r32, n * sizeof(float)));
        TRY(P.alloc((void**)&l.d32, n * sizeof(float)));
        TRY(launch_pack_low(l.G, l.Glow, l.gsc, l.m, D.smooth_prec, s));
        if (l.tc.G) TRY(launch_pack_tc16(l.G, const_cast<void*>(l.tc.G), l.gsc, l.m, D.smooth_prec, s));
        TRY(to_f32(l.dinv32, l.dinv, n, s));
      }
      CHECK(tune_level(P, l, s));
      if (k == 0 && D.fp64_arith == HMG_ARITH_DF64 && df64_supported(D.dim, l.basis.n)) {
        // the finest level's FP64 operator in double-float arithmetic: the factors split once into
        // float pairs (same element-major layout)
        TRY(P.alloc(&l.Gdf, gsz * nc_of(D.dim) * 2 * sizeof(float) + 256));  // prefetch rounding
        TRY(launch_split_df64(l.G, l.Gdf, gsz * nc_of(D.dim), s));
        l.v64 = kApply64Df;
      }
    }
    {
      Phase ph("setup: transfer stencils", s);
      for (size_t k = 0; k + 1 < P.L.size(); ++k)
        for (int a = 0; a < D.dim; ++a) CHECK(build_axis(P, P.L[k], P.L[k + 1], a, &P.L[k].P[a], &P.L[k].PT[a]));
    }
    {
      Phase ph("setup: coarsest dense inverse", s);
      CHECK(build_coarse(P, P.L.back(), s));
    }
    if (D.smoother == HMG_SMOOTH_CHEB) {
      Phase ph("setup: Arnoldi bounds", s);
      for (size_t k = 0; k + 1 < P.L.size(); ++k) CHECK(arnoldi(P, (int)k, s));
    }
    TRY(cudaStreamSynchronize(s));
    return HMG_OK;
  }();
  for (void* t : tmp) dev_free(t, s);
  dev_free(Jstage, s);
  dev_free(bad, s);
  cudaStreamSynchronize(s);  // nothing may still read the host staging vectors
  return st;
}

// ---- graph solves -----------------------------------------------------------------------

// finest-level applies of one V-cycle from a zero guess (the first pre-smoothing step needs none)
long long vcycle_fine_applies(const ProblemImpl& P) {
  if (P.L.size() < 2) return 0;
  const hmg_desc& D = P.desc;
  return (D.nu_pre >= 1 ? D.nu_pre - 1 : 0) + 1 + D.nu_post;
}

// Capture the work `fn` enqueues on s into graph g (appended after nothing: g is empty or a
// body graph); *leaves receives the capture's final dependency set.
template <typename F>
hmg_status capture_into(cudaGraph_t g, cudaStream_t s, F&& fn, std::vector<cudaGraphNode_t>* leaves) {
  TRY(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  hmg_status st = fn();
  if (st == HMG_OK && leaves) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &d, nullptr, &nd);
    if (e == cudaSuccess) leaves->assign(d, d + nd);
    else st = HMG_EDEVICE;
  }
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &out);
  if (st != HMG_OK) return st;
  TRY(e);
  return HMG_OK;
}

hmg_status add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h,
                           cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams prm = {};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  TRY(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &prm));
  *body = prm.conditional.phGraph_out[0];
  return HMG_OK;
}

// One solve of mode `mode` as a graph: prologue, then WHILE(hw){ iteration }. For PCG the
// iteration is [A p, alpha, u, r, ||r||, check] then IF(hi){ z = V(r), beta, p }, so the last
// iteration stops right after the convergence test (Algorithm 1's order).
hmg_status build_graph(ProblemImpl& P, int mode, int cap) {
  if (P.gexec[mode] && P.hist_cap >= cap) return HMG_OK;
  if (P.hist_cap < cap) {
    for (int m = 0; m < 2; ++m) {  // both graphs point at the history array
      if (P.gexec[m]) { cudaGraphExecDestroy(P.gexec[m]); P.gexec[m] = nullptr; }
      if (P.graph[m]) { cudaGraphDestroy(P.graph[m]); P.graph[m] = nullptr; }
    }
    if (!P.cap_stream) TRY(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
    dev_free(P.hist, P.cap_stream);
    P.hist = nullptr;
    pinned_free(P.host_hist, (size_t)(P.hist_cap + 1) * sizeof(double));
    P.host_hist = nullptr;
    TRY(dev_alloc((void**)&P.hist, (cap + 1) * sizeof(double), P.cap_stream));
    TRY(cudaStreamSynchronize(P.cap_stream));
    P.host_hist = static_cast<double*>(pinned_alloc((size_t)(cap + 1) * sizeof(double)));
    if (!P.host_hist) { set_error("pinned host allocation failed"); return HMG_ENOMEM; }
    P.hist_cap = cap;
  }
  if (!P.cap_stream) TRY(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
  cudaStream_t s = P.cap_stream;
  const long long n = P.L[0].m.N;
  cudaGraph_t g = nullptr;
  TRY(cudaGraphCreate(&g, 0));
  P.capturing = true;
  hmg_status st = [&]() -> hmg_status {
    cudaGraphConditionalHandle hw;
    TRY(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
    std::vector<cudaGraphNode_t> leaves;
    double* r = P.pr;
    double* z = P.pz;
    long long c0 = add_launches(0);
    CHECK(capture_into(g, s, [&]() -> hmg_status {
      TRY(cudaMemcpyAsync(r, P.gb, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      TRY(cudaMemsetAsync(P.gu, 0, n * sizeof(double), s));
      CHECK(dot_to(P, r, r, n, FIN_STORE, S_RR0, 0, false, s));
      TRY(start_check(P.S, P.ctrl, P.hist, hw, s));
      if (mode == HMG_MODE_PCG) {
        CHECK(precondition(P, r, z, s));
        TRY(cudaMemcpyAsync(P.pp, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CHECK(dot_to(P, z, r, n, FIN_STORE, S_RHO, 0, false, s));
      }
      return HMG_OK;
    }, &leaves));
    P.gkern[mode][0] = add_launches(0) - c0;
    c0 = add_launches(0);
    cudaGraph_t body;
    CHECK(add_conditional(g, leaves, hw, cudaGraphCondTypeWhile, &body));
    if (mode == HMG_MODE_MG) {
      CHECK(capture_into(body, s, [&]() -> hmg_status {
        CHECK(precondition(P, r, z, s));
        TRY(axpy(P.gu, z, n, 1.0, s));
        TRY(cudaMemcpyAsync(r, P.gb, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        CHECK(apply_level(P, 0, P.gu, r, -1.0, s));
        CHECK(dot_to(P, r, r, n, FIN_STORE, S_RR, 0, false, s));
        TRY(step_check(P.S, P.ctrl, P.hist, hw, hw, 0, s));
        return HMG_OK;
      }, nullptr));
      P.gkern[mode][1] = add_launches(0) - c0;
    } else {
      cudaGraphConditionalHandle hi;
      TRY(cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault));
      std::vector<cudaGraphNode_t> l1;
      CHECK(capture_into(body, s, [&]() -> hmg_status {
        TRY(cudaMemsetAsync(P.ph, 0, n * sizeof(double), s));
        CHECK(apply_level(P, 0, P.pp, P.ph, 1.0, s));
        CHECK(dot_to(P, P.pp, P.ph, n, FIN_STORE, S_PH, 0, false, s));
        TRY(pcg_update(P.gu, r, P.pp, P.ph, n, P.S, P.partial, s));
        TRY(finish(P.partial, n, P.S, FIN_STORE, S_RR, 0, nullptr, s));
        TRY(step_check(P.S, P.ctrl, P.hist, hw, hi, 1, s));
        return HMG_OK;
      }, &l1));
      P.gkern[mode][1] = add_launches(0) - c0;
      c0 = add_launches(0);
      cudaGraph_t rest;
      CHECK(add_conditional(body, l1, hi, cudaGraphCondTypeIf, &rest));
      CHECK(capture_into(rest, s, [&]() -> hmg_status {
        CHECK(precondition(P, r, z, s));
        CHECK(pcg_rho_beta(P, z, r, n, s));
        TRY(pcg_direction(P.pp, z, n, P.S, s));
        return HMG_OK;
      }, nullptr));
      P.gkern[mode][2] = add_launches(0) - c0;
    }
    // capture launched nothing: take the captured kernels back out of the launch count
    add_launches(-(P.gkern[mode][0] + P.gkern[mode][1] + P.gkern[mode][2]));
    cudaGraphExec_t ex = nullptr;
    TRY(cudaGraphInstantiate(&ex, g, 0));
    P.graph[mode] = g;
    P.gexec[mode] = ex;
    return HMG_OK;
  }();
  P.capturing = false;
  if (st != HMG_OK) cudaGraphDestroy(g);
  return st;
}

// ---- lockstep graphs for batched solves ----------------------------------------------------
// Plain graphs (no conditional nodes): PCG: prologue [r = b, u = 0, ||r||, z = V(r), p = z, (z,r)],
// half [h = A p, alpha, u, r, ||r||] and step [z = V(r), beta, p, h = A p, alpha, u, r, ||r||];
// MG: prologue [r = b, u = 0, ||r||] and step [z = V(r), u += z, r = b - A u, ||r||]. Each ends by
// copying ||r_0||^2 and ||r||^2 (slots S_LRR0, S_LRR) into pinned host memory; the host tests convergence between
// launches (Algorithm 1's test position), one synchronization per step for the whole batch.
hmg_status capture_plain(ProblemImpl& P, int mode, int k, cudaStream_t s,
                         const std::function<hmg_status()>& fn) {
  cudaGraph_t g = nullptr;
  const long long c0 = add_launches(0);
  P.capturing = true;
  hmg_status st = HMG_OK;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = fn();
    if (st == HMG_OK) e = cudaMemcpyAsync(P.hostS + 2, P.S + S_LRR0, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e2;
  }
  P.capturing = false;
  P.lkern[mode][k] = add_launches(0) - c0;
  add_launches(-P.lkern[mode][k]);
  if (st != HMG_OK) { if (g) cudaGraphDestroy(g); return st; }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P.lexec[mode][k], g, 0);
  if (g) cudaGraphDestroy(g);
  TRY(e);
  return HMG_OK;
}

hmg_status build_lockstep(ProblemImpl& P, int mode) {
  if (P.lexec[mode][2]) return HMG_OK;
  if (!P.cap_stream) TRY(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
  cudaStream_t s = P.cap_stream;
  const long long n = P.L[0].m.N;
  double* r = P.pr;
  double* z = P.pz;
  auto norm = [&]() -> hmg_status { return dot_to(P, r, r, n, FIN_STORE, S_LRR, 0, false, s); };
  auto apply_update = [&]() -> hmg_status {
    TRY(cudaMemsetAsync(P.ph, 0, n * sizeof(double), s));
    CHECK(apply_level(P, 0, P.pp, P.ph, 1.0, s));
    CHECK(dot_to(P, P.pp, P.ph, n, FIN_STORE, S_PH, 0, false, s));
    TRY(pcg_update(P.gu, r, P.pp, P.ph, n, P.S, P.partial, s));
    TRY(finish(P.partial, n, P.S, FIN_STORE, S_LRR, 0, nullptr, s));
    return HMG_OK;
  };
  CHECK(capture_plain(P, mode, 0, s, [&]() -> hmg_status {
    TRY(cudaMemcpyAsync(r, P.gb, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(cudaMemsetAsync(P.gu, 0, n * sizeof(double), s));
    CHECK(dot_to(P, r, r, n, FIN_STORE, S_LRR0, 0, false, s));
    if (mode == HMG_MODE_PCG) {
      CHECK(precondition(P, r, z, s));
      TRY(cudaMemcpyAsync(P.pp, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CHECK(dot_to(P, z, r, n, FIN_STORE, S_RHO, 0, false, s));
    }
    return HMG_OK;
  }));
  if (mode == HMG_MODE_PCG) {
    CHECK(capture_plain(P, mode, 1, s, [&]() -> hmg_status { return apply_update(); }));
    CHECK(capture_plain(P, mode, 2, s, [&]() -> hmg_status {
      CHECK(precondition(P, r, z, s));
      CHECK(pcg_rho_beta(P, z, r, n, s));
      TRY(pcg_direction(P.pp, z, n, P.S, s));
      return apply_update();
    }));
  } else {
    CHECK(capture_plain(P, mode, 2, s, [&]() -> hmg_status {
      CHECK(precondition(P, r, z, s));
      TRY(axpy(P.gu, z, n, 1.0, s));
      TRY(cudaMemcpyAsync(r, P.gb, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CHECK(apply_level(P, 0, P.gu, r, -1.0, s));
      return norm();
    }));
  }
  return HMG_OK;
}

// Enqueue one graph solve on s (no host synchronization); results land in pinned buffers.
hmg_status graph_solve_enqueue(ProblemImpl& P, int mode, const double* b, double* u, double rtol, int maxit,
                               cudaStream_t s) {
  const int cap = std::max(maxit, 64);
  CHECK(build_graph(P, mode, cap));
  const long long n = P.L[0].m.N;
  TRY(copy_masked(P.gb, b, P.L[0].m, s));
  TRY(set_solve_params(P.S, P.ctrl, rtol, maxit, P.hist_cap, s));
  TRY(cudaGraphLaunch(P.gexec[mode], s));
  TRY(cudaMemcpyAsync(u, P.gu, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TRY(cudaMemcpyAsync(P.host_ctrl, P.ctrl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(P.host_hist, P.hist, (maxit + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  return HMG_OK;
}

// After the stream has completed: iteration count, history and status of a graph solve.
hmg_status graph_solve_finish(ProblemImpl& P, int mode, int* iters, double* res_hist) {
  const int it = P.host_ctrl[0];
  const int status = P.host_ctrl[1];
  if (iters) *iters = it;
  if (res_hist)
    for (int i = 0; i <= it && i <= P.hist_cap; ++i) res_hist[i] = P.host_hist[i];
  // kernels the graph executed: prologue, `it` loop bodies, and (PCG) it-1 second halves
  add_launches(P.gkern[mode][0] + (long long)it * P.gkern[mode][1] +
               (it > 0 ? (long long)(it - 1) * P.gkern[mode][2] : 0));
  const long long v = vcycle_fine_applies(P);
  if (it > 0) P.fine_applies += mode == HMG_MODE_MG ? (long long)it * (v + 1) : v + it + (long long)(it - 1) * v;
  else if (mode == HMG_MODE_PCG && status != ST_NAN) P.fine_applies += v;
  switch (status) {
    case ST_CONVERGED: return HMG_OK;
    case ST_MAXIT: set_error("maximum number of iterations reached"); return HMG_ENOCONV;
    case ST_NAN: set_error("non-finite residual"); return HMG_ENAN;
    default: set_error("graph solve ended in an unexpected state"); return HMG_EDEVICE;
  }
}

// ---- device-memory estimate of a hierarchy (mirrors setup_impl's allocations) -------------
hmg_status estimate_bytes(const hmg_desc& D, size_t* resident, size_t* peak) {
  std::vector<std::pair<std::vector<int>, int>> shapes;
  CHECK(level_shapes(D, shapes));
  const bool mixed = D.smooth_prec != HMG_PREC_FP64;
  std::vector<Mesh> ms;
  for (auto& sh : shapes) ms.push_back(make_mesh(D.dim, sh.first.data(), sh.second));
  size_t res = 0, allocs = 0, max_stage = 0, max_tbuf = 0, arnoldi = 0, blk_temp = 0;
  auto add = [&](size_t b) { res += std::max<size_t>(b, 16); ++allocs; };
  for (size_t k = 0; k < ms.size(); ++k) {
    const Mesh& m = ms[k];
    const size_t gsz = (size_t)(m.nelem * np_of(m)), n = (size_t)m.N;
    add(gsz * nc_of(D.dim) * 8 + 256); add(gsz * 8);
    if (k == 0 && D.fp64_arith == HMG_ARITH_DF64 && df64_supported(D.dim, m.p + 1))
      add(gsz * nc_of(D.dim) * 8 + 256);  // float-pair factors of the double-float operator
    for (int v = 0; v < 5; ++v) add(n * 8);
    if (m.p + 1 <= kMaxNDense && k + 1 < ms.size() && (k == 0 || !mixed))
      add((size_t)m.nelem * np_of(m) * np_of(m) * 8);  // element matrices (dense-apply variant)
    if (D.smoother == HMG_SMOOTH_BLOCKJACOBI && k + 1 < ms.size() && block_size_of(m) > 0) {
      const int mi = block_size_of(m);
      add((size_t)packed_block_doubles(m.nelem, mi) * 8);  // inverted element-interior blocks
      add(n * 8);                                          // D^-1 on shared nodes
      blk_temp = std::max(blk_temp, (size_t)m.nelem * mi * mi * 8 + 512);
    }
    if (mixed) {
      add(low_factor_bytes(m, D.smooth_prec) + 256);
      if (D.smooth_prec != HMG_PREC_FP32) add((size_t)m.nelem * 4);
      if (tc16_supported(m, D.smooth_prec)) {
        add(tc16_phi_bytes(m));
        add(tc16_factor_bytes(m));
      }
      for (int v = 0; v < 5; ++v) add(n * 4);
    }
    max_stage = std::max(max_stage, gsz * D.dim * (D.dim + 1) * 8);
    if (D.smoother == HMG_SMOOTH_CHEB && k + 1 < ms.size())
      arnoldi = std::max(arnoldi, (size_t)(std::min<long long>(D.arnoldi_iters, interior_count(m)) + 1) *
                                      (n + kRedBlocks + 1 + (size_t)D.arnoldi_iters) * 8);
    if (k + 1 < ms.size()) {
      const Mesh& c = ms[k + 1];
      long long od[3] = {c.Nn[0], c.Nn[1], c.Nn[2]};
      for (int a = 0; a < D.dim; ++a) {
        od[a] = m.Nn[a];
        max_tbuf = std::max(max_tbuf, (size_t)(od[0] * od[1] * od[2]));
        const size_t nnz = (size_t)m.Nn[a] * (c.p + 1);
        add((m.Nn[a] + 1) * 4); add(nnz * 4); add(nnz * 8); add(nnz * 4);
        add((c.Nn[a] + 1) * 4); add(nnz * 4); add(nnz * 8); add(nnz * 4);
      }
      long long rd[3] = {m.Nn[0], m.Nn[1], m.Nn[2]};
      for (int a = 0; a < D.dim; ++a) { rd[a] = c.Nn[a]; max_tbuf = std::max(max_tbuf, (size_t)(rd[0] * rd[1] * rd[2])); }
    }
  }
  const long long nI = interior_count(ms.back());
  add((size_t)nI * nI * 8); add((size_t)nI * 8);
  const size_t N0 = (size_t)ms[0].N;
  add(64 * 8); add(4); add(kRedBlocks * 8); add(max_tbuf * 8); add(max_tbuf * 8);
  for (int v = 0; v < 6; ++v) add(N0 * 8);
  add(16);
  res += 1001 * 8;                        // residual history of graph solves (default capacity)
  res += allocs * 512;                    // allocation granularity
  size_t custom = 0;  // setup temporaries of user geometry / coefficient
  const size_t nq0 = (size_t)(ms[0].nelem * np_of(ms[0]));
  if (D.node_xyz) { custom += (size_t)D.dim * N0 * 8; res += (size_t)D.dim * N0 * 8 + 512; }
  if (D.mu_fn) custom += (size_t)(D.dim + 1) * nq0 * 8;
  const size_t temp = std::max(max_stage + 16 + custom + blk_temp,
                               std::max(arnoldi, blocked_gj_work_doubles(nI) * 8 + 1024));
  if (resident) *resident = res;
  if (peak) *peak = res + temp;
  return HMG_OK;
}

bool level_ok(const hmg_problem* p, int level) {
  if (!p || level < 0 || level >= (int)p->impl.L.size()) {
    set_error("invalid problem handle or level");
    return false;
  }
  return true;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

hmg_status hmg_desc_default(hmg_desc* d) {
  if (!d) return HMG_EINVAL;
  memset(d, 0, sizeof(*d));
  d->dim = 3;
  d->nelem[0] = d->nelem[1] = d->nelem[2] = 8;
  d->order = 4;
  d->warp_amp = 0.0;
  d->mu_a = 1.0;
  d->mu_b = 0.0;
  d->mu_k = 2.0;
  d->hier = HMG_HIER_H;
  d->n_hlevels = 3;
  d->smoother = HMG_SMOOTH_CHEB;
  d->nu_pre = 3;
  d->nu_post = 3;
  d->omega = 2.0 / 3.0;
  d->arnoldi_iters = 10;
  d->cheb_lo_frac = 0.25;
  d->cheb_safety = 1.0;
  d->arnoldi_seed = 0;
  d->smooth_prec = HMG_PREC_FP64;
  d->solve_graph = 1;
  d->fp64_arith = HMG_ARITH_FP64;
  d->node_xyz = nullptr;
  d->mu_fn = nullptr;
  d->mu_user = nullptr;
  return HMG_OK;
}

hmg_status hmg_setup(const hmg_desc* desc, void* stream, hmg_problem** out) {
  if (!out) { set_error("null output handle"); return HMG_EINVAL; }
  *out = nullptr;
  CHECK(validate(desc));
  hmg_problem* p = new (std::nothrow) hmg_problem();
  if (!p) { set_error("host allocation failed"); return HMG_ENOMEM; }
  p->impl.desc = *desc;
  if (cudaGetDevice(&p->impl.device) != cudaSuccess) {
    delete p;
    set_error("no CUDA device");
    return HMG_EDEVICE;
  }
  hmg_status st = setup_impl(p->impl, (cudaStream_t)stream);
  if (st != HMG_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    delete p;
    return st;
  }
  p->impl.fine_applies = 0;
  *out = p;
  return HMG_OK;
}

hmg_status hmg_destroy(hmg_problem* p) {
  if (!p) return HMG_OK;
  int cur = 0;
  cudaGetDevice(&cur);
  const int dev = p->impl.device;
  if (cur != dev) cudaSetDevice(dev);
  delete p;
  if (cur != dev) cudaSetDevice(cur);
  return HMG_OK;
}

int hmg_nlevels(const hmg_problem* p) { return p ? (int)p->impl.L.size() : 0; }

size_t hmg_ndof(const hmg_problem* p, int level) {
  if (!level_ok(p, level)) return 0;
  return (size_t)p->impl.L[level].m.N;
}

hmg_status hmg_level_info(const hmg_problem* p, int level, int* nelem3, int* order, size_t* ndof) {
  if (!level_ok(p, level)) return HMG_EINVAL;
  const Mesh& m = p->impl.L[level].m;
  if (nelem3) for (int a = 0; a < 3; ++a) nelem3[a] = m.E[a];
  if (order) *order = m.p;
  if (ndof) *ndof = (size_t)m.N;
  return HMG_OK;
}

size_t hmg_device_bytes(const hmg_problem* p) { return p ? p->impl.bytes : 0; }

hmg_status hmg_level_variants(const hmg_problem* p, int level, int* v_fp64, int* v_vcycle) {
  if (!level_ok(p, level)) return HMG_EINVAL;
  const Level& l = p->impl.L[level];
  if (v_fp64) *v_fp64 = (l.v64 == kApply64Dense && !l.Ke) ? 0 : l.v64;
  if (v_vcycle) *v_vcycle = l.v32;
  return HMG_OK;
}

hmg_status hmg_node_coords(hmg_problem* p, int level, double* xyz, void* stream) {
  if (!level_ok(p, level) || !xyz) { set_error("null argument"); return HMG_EINVAL; }
  const Level& l = p->impl.L[level];
  cudaStream_t s = (cudaStream_t)stream;
  if (p->impl.X0) {  // user geometry: the finest coordinates, or the finest map at this level's nodes
    if (level == 0)
      TRY(cudaMemcpyAsync(xyz, p->impl.X0, (size_t)l.m.dim * l.m.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else
      TRY(launch_level_coords(p->impl.L[0].m, p->impl.L[0].basis, p->impl.X0, l.m, l.basis, xyz, s));
    return HMG_OK;
  }
  TRY(node_coords(xyz, l.m, l.basis.r, p->impl.desc.warp_amp, s));
  return HMG_OK;
}

hmg_status hmg_rhs(hmg_problem* p, const double* f, double* b, void* stream) {
  if (!level_ok(p, 0) || !f || !b) { set_error("null argument"); return HMG_EINVAL; }
  Level& l = p->impl.L[0];
  cudaStream_t s = (cudaStream_t)stream;
  TRY(cudaMemsetAsync(b, 0, l.m.N * sizeof(double), s));
  TRY(launch_mass(l.m, l.basis, f, b, l.wdetJ, s));
  return HMG_OK;
}

hmg_status hmg_apply(hmg_problem* p, int level, const double* x, double* y, void* stream) {
  if (!level_ok(p, level) || !x || !y) { set_error("null argument"); return HMG_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  TRY(cudaMemsetAsync(y, 0, p->impl.L[level].m.N * sizeof(double), s));
  return apply_level(p->impl, level, x, y, 1.0, s);
}

hmg_status hmg_apply_f32(hmg_problem* p, int level, const float* x, float* y, void* stream) {
  if (!level_ok(p, level) || !x || !y) { set_error("null argument"); return HMG_EINVAL; }
  if (!p->impl.L[level].Glow) {
    set_error("the V-cycle operator in FP32 vectors exists only for a smooth_prec other than HMG_PREC_FP64");
    return HMG_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  TRY(cudaMemsetAsync(y, 0, p->impl.L[level].m.N * sizeof(float), s));
  return apply_level(p->impl, level, x, y, 1.0f, s);
}

hmg_status hmg_diag_inv(hmg_problem* p, int level, double* dinv, void* stream) {
  if (!level_ok(p, level) || !dinv) { set_error("null argument"); return HMG_EINVAL; }
  Level& l = p->impl.L[level];
  TRY(cudaMemcpyAsync(dinv, l.dinv, l.m.N * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return HMG_OK;
}

hmg_status hmg_lambda_max(const hmg_problem* p, int level, double* lam) {
  if (!level_ok(p, level) || !lam) { set_error("null argument"); return HMG_EINVAL; }
  *lam = p->impl.L[level].lam;
  return HMG_OK;
}

hmg_status hmg_prolong(hmg_problem* p, int level, const double* xc, double* xf, void* stream) {
  if (!level_ok(p, level) || level + 1 >= (int)p->impl.L.size() || !xc || !xf) {
    set_error("prolongation needs a level with a coarser level below it");
    return HMG_EINVAL;
  }
  return prolong<double>(p->impl, level, xc, xf, false, (cudaStream_t)stream);
}

hmg_status hmg_restrict(hmg_problem* p, int level, const double* rf, double* rc, void* stream) {
  if (!level_ok(p, level) || level + 1 >= (int)p->impl.L.size() || !rf || !rc) {
    set_error("restriction needs a level with a coarser level below it");
    return HMG_EINVAL;
  }
  return restrict_<double>(p->impl, level, rf, rc, (cudaStream_t)stream);
}

hmg_status hmg_smooth(hmg_problem* p, int level, const double* b, double* x, int steps, int zero_guess,
                      void* stream) {
  if (!level_ok(p, level) || !b || !x || steps < 0) { set_error("bad argument"); return HMG_EINVAL; }
  ProblemImpl& P = p->impl;
  Level& l = P.L[level];
  cudaStream_t s = (cudaStream_t)stream;
  if (level == (int)P.L.size() - 1 || (P.desc.smoother == HMG_SMOOTH_CHEB && !(l.lam > 0))) {
    set_error("no smoother on the coarsest level");
    return HMG_EINVAL;
  }
  // caller vectors may carry values on boundary nodes: smooth on masked copies
  TRY(copy_masked(l.b, b, l.m, s));
  if (!zero_guess) TRY(copy_masked(l.x, x, l.m, s));
  CHECK(smooth<double>(P, level, l.b, l.x, steps, zero_guess != 0, s));
  TRY(cudaMemcpyAsync(x, l.x, l.m.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return HMG_OK;
}

hmg_status hmg_vcycle(hmg_problem* p, const double* r, double* z, void* stream) {
  if (!level_ok(p, 0) || !r || !z) { set_error("null argument"); return HMG_EINVAL; }
  ProblemImpl& P = p->impl;
  cudaStream_t s = (cudaStream_t)stream;
  TRY(copy_masked(P.pr, r, P.L[0].m, s));
  return precondition(P, P.pr, z, s);
}

// z = M^-1 r of a solve that does not take the problem's own V-cycle (nullptr: the V-cycle)
using Precond = std::function<hmg_status(const double* r, double* z)>;
static hmg_status solve_impl(hmg_problem* p, int mode, const double* b, double* u, double rtol, int maxit,
                             int* iters, double* res_hist, void* stream, const Precond& pre = nullptr);

// Reads (and clears) the device error flag set by bounded waits inside kernels.
static hmg_status device_error(ProblemImpl& P, cudaStream_t s) {
  int h = 0;
  TRY(cudaMemcpyAsync(&h, P.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (h != 0) {
    TRY(cudaMemsetAsync(P.err, 0, sizeof(int), s));
    set_error("a bounded wait inside a kernel gave up (error code " + std::to_string(h) + ")");
    return HMG_ETIMEOUT;
  }
  return HMG_OK;
}

hmg_status hmg_solve(hmg_problem* p, int mode, const double* b, double* u, double rtol, int maxit, int* iters,
                     double* res_hist, void* stream) {
  hmg_status st;
  if (p && p->impl.desc.solve_graph && (mode == HMG_MODE_MG || mode == HMG_MODE_PCG) && b && u && maxit >= 0 &&
      rtol >= 0.0) {
    cudaStream_t s = (cudaStream_t)stream;
    Phase ph(mode == HMG_MODE_PCG ? "solve (PCG graph)" : "solve (MG graph)", s);
    st = graph_solve_enqueue(p->impl, mode, b, u, rtol, maxit, s);
    if (st == HMG_OK) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { set_error(std::string("graph solve: ") + cudaGetErrorString(e)); return HMG_EDEVICE; }
      st = graph_solve_finish(p->impl, mode, iters, res_hist);
    }
  } else {
    st = solve_impl(p, mode, b, u, rtol, maxit, iters, res_hist, stream);
  }
  if (p && (st == HMG_OK || st == HMG_ENOCONV || st == HMG_ENAN)) {
    hmg_status de = device_error(p->impl, (cudaStream_t)stream);
    if (de != HMG_OK) return de;
  }
  return st;
}

hmg_status hmg_solve_low_order(hmg_problem* p, hmg_problem* low, const double* b, double* u, double rtol,
                               int maxit, double inner_rtol, int* iters, long long* inner_iters, double* res_hist,
                               void* stream) {
  if (!level_ok(p, 0) || !level_ok(low, 0) || p == low) { set_error("bad problem handles"); return HMG_EINVAL; }
  const Mesh& mh = p->impl.L[0].m;
  const Mesh& ml = low->impl.L[0].m;
  bool same = mh.dim == ml.dim && ml.p == 1;
  for (int a = 0; a < mh.dim; ++a) same = same && ml.Nn[a] == mh.Nn[a];
  if (!same) {
    set_error("the low-order problem must be of order 1 on the same node grid (nelem = order * nelem)");
    return HMG_EINVAL;
  }
  if (!(inner_rtol > 0.0) || !(inner_rtol < 1.0)) { set_error("inner_rtol must be in (0, 1)"); return HMG_EINVAL; }
  long long inner = 0;
  if (inner_iters) *inner_iters = 0;
  // M^-1 r: the low-order system solved by its own multigrid-preconditioned CG to inner_rtol
  Precond pre = [&](const double* r, double* z) -> hmg_status {
    int it = 0;
    const hmg_status st = hmg_solve(low, HMG_MODE_PCG, r, z, inner_rtol, 10000, &it, nullptr, stream);
    inner += it;
    if (st != HMG_OK) {
      set_error(std::string("low-order solve: ") + hmg_last_error());
      return st == HMG_ENOCONV ? HMG_ENOCONV : st;
    }
    return HMG_OK;
  };
  hmg_status st = solve_impl(p, HMG_MODE_PCG, b, u, rtol, maxit, iters, res_hist, stream, pre);
  if (inner_iters) *inner_iters = inner;
  if (st == HMG_OK || st == HMG_ENOCONV || st == HMG_ENAN) {
    hmg_status de = device_error(p->impl, (cudaStream_t)stream);
    if (de != HMG_OK) return de;
  }
  return st;
}

// Two finest-level FP64 vectors for hmg_apply_host / hmg_solve_host, allocated from the stream-ordered
// pool on the first such call and held until hmg_destroy.
static hmg_status host_staging(ProblemImpl& P, cudaStream_t s) {
  if (P.hx) return HMG_OK;
  const size_t nb = (size_t)P.L[0].m.N * sizeof(double);
  TRY(dev_alloc((void**)&P.hx, nb, s));
  P.dev_allocs.push_back(P.hx);
  TRY(dev_alloc((void**)&P.hy, nb, s));
  P.dev_allocs.push_back(P.hy);
  return HMG_OK;
}

hmg_status hmg_apply_host(hmg_problem* p, int level, const double* x_host, double* y_host, void* stream) {
  if (!level_ok(p, level) || !x_host || !y_host) { set_error("null argument"); return HMG_EINVAL; }
  ProblemImpl& P = p->impl;
  cudaStream_t s = (cudaStream_t)stream;
  CHECK(host_staging(P, s));
  const size_t nb = (size_t)P.L[level].m.N * sizeof(double);
  TRY(cudaMemcpyAsync(P.hx, x_host, nb, cudaMemcpyHostToDevice, s));
  TRY(cudaMemsetAsync(P.hy, 0, nb, s));
  CHECK(apply_level(P, level, P.hx, P.hy, 1.0, s));
  TRY(cudaMemcpyAsync(y_host, P.hy, nb, cudaMemcpyDeviceToHost, s));
  return device_error(P, s);  // synchronizes s
}

hmg_status hmg_solve_host(hmg_problem* p, int mode, const double* f_host, double* u_host, double rtol, int maxit,
                          int* iters, double* res_hist, void* stream) {
  if (!level_ok(p, 0) || !f_host || !u_host) { set_error("null argument"); return HMG_EINVAL; }
  ProblemImpl& P = p->impl;
  cudaStream_t s = (cudaStream_t)stream;
  CHECK(host_staging(P, s));
  const size_t nb = (size_t)P.L[0].m.N * sizeof(double);
  TRY(cudaMemcpyAsync(P.hx, f_host, nb, cudaMemcpyHostToDevice, s));
  CHECK(hmg_rhs(p, P.hx, P.hy, stream));                 // b = M f into hy
  const hmg_status st = hmg_solve(p, mode, P.hy, P.hx, rtol, maxit, iters, res_hist, stream);
  if (st != HMG_OK && st != HMG_ENOCONV && st != HMG_ENAN) return st;
  TRY(cudaMemcpyAsync(u_host, P.hx, nb, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  return st;
}

static hmg_status solve_impl(hmg_problem* p, int mode, const double* b, double* u, double rtol, int maxit,
                             int* iters, double* res_hist, void* stream, const Precond& pre) {
  if (!level_ok(p, 0) || !b || !u || maxit < 0 || !(rtol >= 0.0)) { set_error("bad argument"); return HMG_EINVAL; }
  if (mode != HMG_MODE_MG && mode != HMG_MODE_PCG) { set_error("bad mode"); return HMG_EINVAL; }
  ProblemImpl& P = p->impl;
  cudaStream_t s = (cudaStream_t)stream;
  const Level& l0 = P.L[0];
  const long long n = l0.m.N;
  double* r = P.pr;
  double* z = P.pz;
  if (iters) *iters = 0;
  TRY(cudaMemsetAsync(u, 0, n * sizeof(double), s));
  TRY(copy_masked(r, b, l0.m, s));
  CHECK(dot_to(P, r, r, n, FIN_STORE, S_RR0, 0, true, s));
  TRY(cudaStreamSynchronize(s));
  const double r0 = sqrt(*P.hostS);
  if (!isfinite(r0)) { set_error("non-finite right-hand side"); return HMG_ENAN; }
  if (res_hist) res_hist[0] = r0;
  if (r0 == 0.0) return HMG_OK;
  const double tol = rtol * r0;
  if (mode == HMG_MODE_MG) {
    double* bm = P.ph;  // masked copy of b
    TRY(cudaMemcpyAsync(bm, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    for (int it = 1; it <= maxit; ++it) {
      CHECK(pre ? pre(r, z) : precondition(P, r, z, s));  // z = B (b - A u)
      TRY(axpy(u, z, n, 1.0, s));       // u += z
      TRY(cudaMemcpyAsync(r, bm, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CHECK(apply_level(P, 0, u, r, -1.0, s));
      CHECK(dot_to(P, r, r, n, FIN_STORE, S_RR, 0, true, s));
      TRY(cudaStreamSynchronize(s));
      const double rn = sqrt(*P.hostS);
      if (res_hist) res_hist[it] = rn;
      if (iters) *iters = it;
      if (!isfinite(rn)) { set_error("non-finite residual"); return HMG_ENAN; }
      if (rn <= tol) return HMG_OK;
    }
    set_error("maximum number of V-cycles reached");
    return HMG_ENOCONV;
  }
  // PCG (Algorithm 1, read as standard preconditioned CG from u0 = 0)
  double* pp = P.pp;
  double* h = P.ph;
  CHECK(pre ? pre(r, z) : precondition(P, r, z, s));
  TRY(cudaMemcpyAsync(pp, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CHECK(dot_to(P, z, r, n, FIN_STORE, S_RHO, 0, false, s));
  for (int it = 1; it <= maxit; ++it) {
    TRY(cudaMemsetAsync(h, 0, n * sizeof(double), s));
    CHECK(apply_level(P, 0, pp, h, 1.0, s));
    CHECK(dot_to(P, pp, h, n, FIN_STORE, S_PH, 0, false, s));
    TRY(pcg_update(u, r, pp, h, n, P.S, P.partial, s));
    TRY(finish(P.partial, n, P.S, FIN_STORE, S_RR, 0, P.hostS, s));
    TRY(cudaStreamSynchronize(s));
    const double rn = sqrt(*P.hostS);
    if (res_hist) res_hist[it] = rn;
    if (iters) *iters = it;
    if (!isfinite(rn)) { set_error("non-finite residual"); return HMG_ENAN; }
    if (rn <= tol) return HMG_OK;
    CHECK(pre ? pre(r, z) : precondition(P, r, z, s));
    CHECK(pcg_rho_beta(P, z, r, n, s));
    TRY(pcg_direction(pp, z, n, P.S, s));
  }
  set_error("maximum number of PCG iterations reached");
  return HMG_ENOCONV;
}

hmg_status hmg_solve_batched(hmg_problem* const* probs, int n, int mode, const double* const* b,
                             double* const* u, double rtol, int maxit, int* iters, double* const* res_hist,
                             int* status, void* stream) {
  if (!probs || n < 0 || !b || !u || maxit < 0 || !(rtol >= 0.0) || (mode != HMG_MODE_MG && mode != HMG_MODE_PCG)) {
    set_error("bad argument");
    return HMG_EINVAL;
  }
  if (n == 0) return HMG_OK;
  for (int i = 0; i < n; ++i) {
    if (!level_ok(probs[i], 0) || !b[i] || !u[i]) { set_error("bad problem handle or vector in the batch"); return HMG_EINVAL; }
    for (int j = 0; j < i; ++j)
      if (probs[j] == probs[i]) { set_error("a handle appears twice in the batch"); return HMG_EINVAL; }
  }
  // grouped batch plan (one graph for all problems) unless a problem has no grouped form or
  // HMG_BATCH_LOCKSTEP=1 asks for per-problem graphs in lockstep
  static const bool lockstep_only = [] {
    const char* v = getenv("HMG_BATCH_LOCKSTEP");
    return v && v[0] == '1';
  }();
  bool grouped = !lockstep_only;
  for (int i = 0; i < n && grouped; ++i) grouped = batch_supported(probs[i]);
  if (grouped) {
    hmg_batch* plan = nullptr;
    CHECK(hmg_batch_create(probs, n, mode, std::max(maxit, 64), &plan));
    const hmg_status st = hmg_batch_solve(plan, b, u, rtol, maxit, iters, res_hist, status, stream);
    const std::string msg = hmg_last_error();
    hmg_batch_destroy(plan);
    if (st != HMG_OK) set_error(msg);
    return st;
  }
  for (int i = 0; i < n; ++i) CHECK(build_lockstep(probs[i]->impl, mode));
  // streams in the fan-out (HMG_BATCH_STREAMS, 1..64, default 32)
  static const int K = [] {
    const char* v = getenv("HMG_BATCH_STREAMS");
    const int k = v ? atoi(v) : 32;
    return k < 1 ? 1 : (k > 64 ? 64 : k);
  }();
  static std::mutex pool_mu;
  static std::vector<cudaStream_t> pool[64];
  int dev = 0;
  TRY(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(pool_mu);
    if (dev >= 0 && dev < 64 && pool[dev].empty())
      for (int k = 0; k < K; ++k) {
        cudaStream_t sk;
        TRY(cudaStreamCreateWithFlags(&sk, cudaStreamNonBlocking));
        pool[dev].push_back(sk);
      }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int used = std::min(n, K);
  std::vector<cudaEvent_t> ev(used + 1, nullptr);
  for (auto& e : ev) TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  std::vector<int> it(n, 0), st(n, 1);  // st: 1 running, 0 converged, -3 maxit, -7 nan
  std::vector<double> r0(n, 0.0);
  auto hist_set = [&](int i, int k, double v) { if (res_hist && res_hist[i]) res_hist[i][k] = v; };
  // launch `k`-graphs of the problems in `which` over the pool, then join on s and synchronize
  double t_enqueue = 0.0, t_wait = 0.0;  // host seconds (HMG_TRACE=1 prints them)
  int nsteps = 0;
  auto step = [&](const std::vector<int>& which, int k0, int k1) -> hmg_status {
    const auto c0 = std::chrono::steady_clock::now();
    TRY(cudaEventRecord(ev[used], s));
    for (int q = 0; q < used; ++q) TRY(cudaStreamWaitEvent(pool[dev][q], ev[used], 0));
    for (size_t w = 0; w < which.size(); ++w) {
      const int i = which[w];
      ProblemImpl& P = probs[i]->impl;
      cudaStream_t si = pool[dev][i % K];
      if (k0 == 0) {
        TRY(copy_masked(P.gb, b[i], P.L[0].m, si));
      }
      for (int k = k0; k <= k1; ++k) {
        if (!P.lexec[mode][k]) continue;
        TRY(cudaGraphLaunch(P.lexec[mode][k], si));
        add_launches(P.lkern[mode][k]);
      }
    }
    for (int q = 0; q < used; ++q) {
      TRY(cudaEventRecord(ev[q], pool[dev][q]));
      TRY(cudaStreamWaitEvent(s, ev[q], 0));
    }
    const auto c1 = std::chrono::steady_clock::now();
    TRY(cudaStreamSynchronize(s));
    const auto c2 = std::chrono::steady_clock::now();
    t_enqueue += std::chrono::duration<double>(c1 - c0).count();
    t_wait += std::chrono::duration<double>(c2 - c1).count();
    ++nsteps;
    return HMG_OK;
  };
  hmg_status err = [&]() -> hmg_status {
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    // prologue (+ PCG's first half-iteration unless maxit == 0)
    CHECK(step(all, 0, (mode == HMG_MODE_PCG && maxit > 0) ? 1 : 0));
    std::vector<int> active;
    auto check = [&](int i) {
      ProblemImpl& P = probs[i]->impl;
      const double rn = sqrt(P.hostS[3]);
      hist_set(i, it[i], rn);
      if (!std::isfinite(rn)) st[i] = -7;
      else if (rn <= rtol * r0[i]) st[i] = 0;
      else if (it[i] >= maxit) st[i] = -3;
    };
    for (int i = 0; i < n; ++i) {
      ProblemImpl& P = probs[i]->impl;
      r0[i] = sqrt(P.hostS[2]);
      hist_set(i, 0, r0[i]);
      if (!std::isfinite(r0[i])) { st[i] = -7; continue; }
      if (r0[i] == 0.0) { st[i] = 0; continue; }
      if (maxit == 0) { st[i] = -3; continue; }
      if (mode == HMG_MODE_PCG) {
        it[i] = 1;
        check(i);
      }
      if (st[i] == 1) active.push_back(i);
    }
    while (!active.empty()) {
      CHECK(step(active, 2, 2));
      std::vector<int> next;
      for (int i : active) {
        ++it[i];
        check(i);
        if (st[i] == 1) next.push_back(i);
      }
      active.swap(next);
    }
    for (int i = 0; i < n; ++i) {
      ProblemImpl& P = probs[i]->impl;
      if (r0[i] == 0.0 || !std::isfinite(r0[i]) || maxit == 0)
        TRY(cudaMemsetAsync(u[i], 0, P.L[0].m.N * sizeof(double), s));
      else
        TRY(cudaMemcpyAsync(u[i], P.gu, P.L[0].m.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    TRY(cudaStreamSynchronize(s));
    return HMG_OK;
  }();
  for (auto& e : ev) cudaEventDestroy(e);
  if (Phase::timing())
    fprintf(stderr, "hmg batched: %d problems, %d steps, host enqueue %.3f s, wait for the device %.3f s\n", n,
            nsteps, t_enqueue, t_wait);
  if (err != HMG_OK) return err;
  hmg_status first = HMG_OK;
  for (int i = 0; i < n; ++i) {
    ProblemImpl& P = probs[i]->impl;
    const long long v = vcycle_fine_applies(P);
    if (it[i] > 0) P.fine_applies += mode == HMG_MODE_MG ? (long long)it[i] * (v + 1) : v + it[i] + (long long)(it[i] - 1) * v;
    hmg_status si = st[i] == 0 ? HMG_OK : (st[i] == -3 ? HMG_ENOCONV : HMG_ENAN);
    if (si == HMG_OK) si = device_error(P, s);
    if (iters) iters[i] = it[i];
    if (status) status[i] = si;
    if (first == HMG_OK && si != HMG_OK) first = si;
  }
  if (first == HMG_ENOCONV) set_error("maximum number of iterations reached in the batch");
  if (first == HMG_ENAN) set_error("non-finite residual in the batch");
  return first;
}

size_t hmg_desc_ndof(const hmg_desc* d) {
  if (validate(d) != HMG_OK) return 0;
  size_t n = 1;
  for (int a = 0; a < d->dim; ++a) n *= (size_t)d->nelem[a] * d->order + 1;
  return n;
}

hmg_status hmg_estimate_bytes(const hmg_desc* d, size_t* resident, size_t* peak) {
  CHECK(validate(d));
  return estimate_bytes(*d, resident, peak);
}

long long hmg_fine_applies(const hmg_problem* p) { return p ? p->impl.fine_applies : 0; }

long long hmg_launch_count(void) { return add_launches(0); }

const char* hmg_status_string(hmg_status s) {
  switch (s) {
    case HMG_OK: return "ok";
    case HMG_EINVAL: return "invalid argument";
    case HMG_ENOMEM: return "out of memory";
    case HMG_ENOCONV: return "not converged";
    case HMG_EDEVICE: return "CUDA error";
    case HMG_ETIMEOUT: return "timed out";
    case HMG_EBUSY: return "busy";
    case HMG_ENAN: return "non-finite value";
  }
  return "unknown status";
}

const char* hmg_last_error(void) { return g_err.c_str(); }

hmg_status hmg_selftest_bounded_wait(unsigned polls, int* timed_out) {
  if (!timed_out || polls == 0 || polls > (1u << 24)) { set_error("polls must be in 1..2^24"); return HMG_EINVAL; }
  int* d = nullptr;
  TRY(cudaMalloc((void**)&d, sizeof(int)));
  cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
  if (e == cudaSuccess) e = bounded_wait_probe(polls, d, 0);
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  TRY(e);
  *timed_out = h;
  return h == 1 ? HMG_ETIMEOUT : HMG_OK;
}

hmg_status hmg_host_basis(int order, double* gll, double* gx, double* gw) {
  if (order < 1 || order > 16) { set_error("order must be in 1..16"); return HMG_EINVAL; }
  Basis1D b;
  make_basis(order, &b);
  for (int i = 0; i <= order; ++i) {
    if (gll) gll[i] = b.r[i];
    if (gx) gx[i] = b.g[i];
    if (gw) gw[i] = b.w[i];
  }
  return HMG_OK;
}

hmg_status hmg_host_hessenberg_max_real_eig(const double* H, int m, double* out) {
  if (!H || !out || m < 1) { set_error("bad argument"); return HMG_EINVAL; }
  *out = hessenberg_max_real_eig(H, m);
  return isfinite(*out) ? HMG_OK : HMG_ENOCONV;
}

}  // extern "C"
