// hmg_restrict_noalloc: the residual restriction r_c = P^T r_f for callers that cannot
// allocate device memory -- code that runs where cudaMalloc is forbidden or unsafe (inside
// a real-time loop with an allocation ban, under a memory manager that owns the whole
// device, in a plug-in that may only use memory its host hands in) and therefore cannot
// create an hmg_problem, whose setup allocates the hierarchy.
//
// It needs no handle: the 1D transfer stencils are computed on the host from the mesh
// sizes and orders, and both the stencils and the intermediate arrays of the per-axis
// passes live in the fixed file-scope device arrays below. The passes are the same
// kernel that hmg_restrict launches (axis_pass / k_axis).
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "vector.cuh"

namespace hmg {

namespace {

// Fixed device storage, held by every device that loads the library until the process exits.
constexpr long long kScratchDoubles = 2LL << 20;      // 16 MiB: both intermediate passes
constexpr int kMaxAxisNodes = 4097;                    // nodes per axis of the fine mesh
constexpr int kMaxAxisEntries = kMaxAxisNodes * kMaxN; // stencil entries per axis

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];
static __device__ __align__(256) int g_noalloc_rowptr[3][kMaxAxisNodes + 1];
static __device__ __align__(256) int g_noalloc_col[3][kMaxAxisEntries];
static __device__ __align__(256) double g_noalloc_val[3][kMaxAxisEntries];

struct DeviceSymbols {
  bool ready = false;
  double* scratch = nullptr;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
};

constexpr int kMaxDevices = 64;
std::mutex g_sym_mu;
DeviceSymbols g_sym[kMaxDevices];

// Device addresses of the fixed arrays on the current device (looked up once per device;
// host code must never hand the arrays' host-side names to a kernel).
cudaError_t symbols(DeviceSymbols** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_sym_mu);
  DeviceSymbols& s = g_sym[dev];
  if (!s.ready) {
    if ((e = cudaGetSymbolAddress((void**)&s.scratch, g_noalloc_scratch)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.rowptr, g_noalloc_rowptr)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.col, g_noalloc_col)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void**)&s.val, g_noalloc_val)) != cudaSuccess) return e;
    s.ready = true;
  }
  *out = &s;
  return cudaSuccess;
}

// Rows = coarse nodes along one axis; entry (I, v): fine node I with v = coarse basis
// function at that node's reference coordinate (the transpose of P_ij = phi_j(p_i)).
void restriction_stencil(int Ef, int pf, int Ec, int pc, std::vector<int>& rowptr, std::vector<int>& col,
                         std::vector<double>& val) {
  Basis1D bf, bc;
  make_basis(pf, &bf);
  make_basis(pc, &bc);
  const int ratio = Ef / Ec;
  const int nf = Ef * pf + 1, ncn = Ec * pc + 1;
  std::vector<std::vector<std::pair<int, double>>> rows(ncn);
  double v[kMaxN];
  for (int I = 0; I < nf; ++I) {
    const int ef = I / pf < Ef - 1 ? I / pf : Ef - 1;
    const int i = I - ef * pf;
    const int ec = ef / ratio;
    lagrange_row(bc.r, pc + 1, ((ef % ratio) + bf.r[i]) / ratio, v);
    for (int k = 0; k <= pc; ++k)
      if (v[k] != 0.0) rows[ec * pc + k].push_back({I, v[k]});
  }
  rowptr.assign(1, 0);
  col.clear();
  val.clear();
  for (auto& r : rows) {
    for (auto& e : r) {
      col.push_back(e.first);
      val.push_back(e.second);
    }
    rowptr.push_back((int)col.size());
  }
}

}  // namespace

}  // namespace hmg

using namespace hmg;

extern "C" hmg_status hmg_restrict_noalloc(int dim, const int nelem_fine[3], int order_fine, int order_coarse,
                                           int halve_mesh, const double* rf_dev, double* rc_dev, void* stream) {
  if ((dim != 2 && dim != 3) || !nelem_fine || !rf_dev || !rc_dev) {
    set_error("hmg_restrict_noalloc: bad dim or null pointer");
    return HMG_EINVAL;
  }
  if (order_fine < 1 || order_fine > 16 || order_coarse < 1 || order_coarse > order_fine) {
    set_error("hmg_restrict_noalloc: orders must satisfy 1 <= order_coarse <= order_fine <= 16");
    return HMG_EINVAL;
  }
  if (!halve_mesh && order_coarse == order_fine) {
    set_error("hmg_restrict_noalloc: the coarse level must halve the mesh or lower the order");
    return HMG_EINVAL;
  }
  int Ef[3] = {1, 1, 1}, Ec[3] = {1, 1, 1};
  long long nf[3] = {1, 1, 1}, nc[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) {
    Ef[a] = nelem_fine[a];
    if (Ef[a] < 1 || (halve_mesh && Ef[a] % 2)) {
      set_error("hmg_restrict_noalloc: elements per axis must be >= 1 (and even when halving the mesh)");
      return HMG_EINVAL;
    }
    Ec[a] = halve_mesh ? Ef[a] / 2 : Ef[a];
    nf[a] = (long long)Ef[a] * order_fine + 1;
    nc[a] = (long long)Ec[a] * order_coarse + 1;
    if (nf[a] > kMaxAxisNodes) {
      set_error("hmg_restrict_noalloc: more than " + std::to_string(kMaxAxisNodes) +
                " fine nodes along an axis (fixed stencil storage)");
      return HMG_EINVAL;
    }
  }
  // intermediates of the passes along x, then y: (nc0, nf1, nf2) and (nc0, nc1, nf2)
  const long long need1 = nc[0] * nf[1] * nf[2];
  const long long need2 = dim == 3 ? nc[0] * nc[1] * nf[2] : 0;
  if (need1 + need2 > kScratchDoubles) {
    set_error("hmg_restrict_noalloc: the intermediate passes need " + std::to_string(need1 + need2) +
              " doubles; the fixed scratch holds " + std::to_string(kScratchDoubles));
    return HMG_EINVAL;
  }
  DeviceSymbols* sym = nullptr;
  cudaError_t e = symbols(&sym);
  if (e != cudaSuccess) {
    set_error(std::string("hmg_restrict_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return HMG_EDEVICE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Axis1D ax[3];
  for (int a = 0; a < dim; ++a) {
    std::vector<int> rp, ci;
    std::vector<double> v;
    restriction_stencil(Ef[a], order_fine, Ec[a], order_coarse, rp, ci, v);
    // pageable host sources: each copy has finished reading them when it returns
    e = cudaMemcpyAsync(sym->rowptr + a * (kMaxAxisNodes + 1), rp.data(), rp.size() * sizeof(int),
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sym->col + (size_t)a * kMaxAxisEntries, ci.data(), ci.size() * sizeof(int),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sym->val + (size_t)a * kMaxAxisEntries, v.data(), v.size() * sizeof(double),
                          cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      set_error(std::string("hmg_restrict_noalloc: stencil upload: ") + cudaGetErrorString(e));
      return HMG_EDEVICE;
    }
    ax[a].n_out = (int)nc[a];
    ax[a].n_in = (int)nf[a];
    ax[a].rowptr = sym->rowptr + a * (kMaxAxisNodes + 1);
    ax[a].col = sym->col + (size_t)a * kMaxAxisEntries;
    ax[a].val = sym->val + (size_t)a * kMaxAxisEntries;
    ax[a].val32 = nullptr;
  }
  // every entry of each intermediate and of rc is written by its pass: nothing to clear
  double* bufs[2] = {sym->scratch, sym->scratch + need1};
  long long od[3] = {nf[0], nf[1], nf[2]};
  const double* in = rf_dev;
  for (int a = 0; a < dim; ++a) {
    od[a] = nc[a];
    const bool last = a == dim - 1;
    double* out = last ? rc_dev : bufs[a & 1];
    e = axis_pass<double>(in, out, od, a, ax[a], a == 0, last, 0, s);
    if (e != cudaSuccess) {
      set_error(std::string("hmg_restrict_noalloc: ") + cudaGetErrorString(e));
      return HMG_EDEVICE;
    }
    in = out;
  }
  return HMG_OK;
}
