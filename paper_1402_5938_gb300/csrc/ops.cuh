// Host launchers of the element kernels, dispatched from the runtime order p to the
// compile-time node count N = p + 1 (2..17).
#pragma once

#include <vector>

#include "common.cuh"

namespace hmg {

// y += alpha * A x in FP64 (G [E][NC][NP] in FP64). Variant 3 stages G with bulk TMA copies (when
// the slab fits in shared memory) and needs G allocated with >= 16 bytes of tail padding; a
// timed-out wait sets *err (device int) to a nonzero code. `variant` selects the form (0..3
// point-parallel block shapes, 3 = TMA-staged G; 4 dense; 5, 6 pencil, below); setup picks it per
// level by timing (autotuning).
// FP64 variant kApply64Dense: stored element matrices Ke (launch_elem_mats) instead of sum
// factorization, for orders with N <= kMaxNDense; other variants ignore Ke.
constexpr int kApply64Dense = 4;
constexpr int kMaxNDense = 3;
// FP64 variants 5 and 6: the pencil form (one thread per element line, even/odd line products from
// order 4 on) in FP64 arithmetic on G as stored, factors read at their use (5) or one phase ahead
// (6, orders with N <= kPencil64AheadMaxN).
constexpr int kApply64Pencil = 5;
constexpr int kApply64PencilAhead = 6;
constexpr int kPencil64AheadMaxN = 9;
// Whether the FP64 pencil form's tile (4 or 3 buffers of EPB elements in FP64) fits a block's
// shared memory (not at 3D N = 15, 16).
bool pencil64_fits(int dim, int n);
// The FP64 variants a level can run: 0-3, 4 with element matrices, and from order 7 on (where
// its even/odd products save enough to compete; measured slower at order 4, equal at order 2)
// 5 where the pencil tile fits and 6 for N <= 9.
constexpr int kPencil64MinN = 8;
inline std::vector<int> apply64_variants(int dim, int n, bool has_ke) {
  std::vector<int> v = {0, 1, 2, 3};
  if (has_ke) v.push_back(kApply64Dense);
  if (n >= kPencil64MinN && pencil64_fits(dim, n)) {
    v.push_back(kApply64Pencil);
    if (n <= kPencil64AheadMaxN) v.push_back(kApply64PencilAhead);
  }
  return v;
}
// FP64 variant kApply64Df: the FP64 operator (FP64 vectors, the FP64 factors split once into
// float pairs, Gdf) in double-float arithmetic (df64.cuh, about 48 significant bits), the pencil
// form with factors read at their use; for orders with N <= kDf64MaxN where the tile fits. Never
// chosen by timing: a problem asks for it (hmg_desc.fp64_arith) on its finest level.
constexpr int kApply64Df = 7;
constexpr int kDf64MaxN = 9;
bool df64_supported(int dim, int n);
cudaError_t launch_apply_df64(const Mesh& m, const Basis1D& b, const double* x, double* y, const void* Gdf,
                              double alpha, cudaStream_t s);
// Gdf[i] = (hi, lo) float pair of G[i] (n values; Gdf holds n float2 and >= 256 bytes more)
cudaError_t launch_split_df64(const double* G, void* Gdf, long long n, cudaStream_t s);
cudaError_t launch_apply_f64(const Mesh& m, const Basis1D& b, const double* x, double* y,
                             const double* G, double alpha, int* err, cudaStream_t s, int variant = 0,
                             const double* Ke = nullptr, const void* Gdf = nullptr);
// Ke[(e * NP + b) * NP + a] = K_e[a][b], the element stiffness matrices (all nodes; the apply
// masks the boundary), by sum-factorized unit columns.
cudaError_t launch_elem_mats(const Mesh& m, const Basis1D& b, const double* G, double* Ke, cudaStream_t s);
// The operator of the mixed V-cycle, y += alpha * A x with FP32 vectors and arithmetic (the pencil
// form of pencil.cuh) and geometric factors Glow in precision prec: HMG_PREC_FP32, or 16 bits
// (HMG_PREC_FP16 / HMG_PREC_BF16, stored divided by the per-element powers of two gsc), in the
// grouped layout launch_pack_low writes (low_factor_bytes bytes; allocate >= 256 bytes more for
// the L2 prefetches' rounding). variant 0 loads a thread's factors one phase before the pointwise
// product, 1 before the first phase (small orders; as 0 otherwise), 2 at their use; variant
// kApplyLowTc (16-bit factors, 3D, orders <= kTc16MaxN - 1) is the tensor-core form of tc16.cuh,
// which needs *tc and the device error flag err (set by a timed-out wait). Setup picks the
// variant per level by timing.
constexpr int kApplyLowVariants = 3;
constexpr int kApplyLowTc = 3;
constexpr int kTc16MaxN = 5;
// Data of the tensor-core form: the factors in its own layout (tc16_factor_bytes, written by
// launch_pack_tc16), the reference gradient image (tc16_phi_image, tc16_phi_bytes) and the
// power of two applied to v.
struct Tc16Data {
  const void* G = nullptr;
  const void* phi = nullptr;
  float vsc = 1.0f;
};
size_t low_factor_bytes(const Mesh& m, int prec);
cudaError_t launch_apply_low(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* Glow,
                             const float* gsc, float alpha, int prec, cudaStream_t s, int variant = 0,
                             const Tc16Data* tc = nullptr, int* err = nullptr);
// Glow (zero-filled beforehand) from G [E][NC][NP] in FP64; 16-bit precisions also write gsc[e].
cudaError_t launch_pack_low(const double* G, void* Glow, float* gsc, const Mesh& m, int prec, cudaStream_t s);
// The tensor-core form is built only with HMG_TC16=1 in the environment (opt-in): it
// measured slower than the pencil form on every level it supports, and building it costs a second
// copy of the factors and autotuning time at setup.
bool tc16_enabled();
bool tc16_supported(const Mesh& m, int prec);
size_t tc16_phi_bytes(const Mesh& m);
size_t tc16_factor_bytes(const Mesh& m);
void tc16_phi_image(const Basis1D& b, std::vector<unsigned char>& img, float* vsc);
// The tensor-core layout of the 16-bit factors (zero-filled beforehand); writes gsc[e] as
// launch_pack_low does.
cudaError_t launch_pack_tc16(const double* G, void* Gtc, float* gsc, const Mesh& m, int prec, cudaStream_t s);

// Geometry, stage 1: Gauss-point coordinates and Jacobians into the stage buffer
// J [E][dim*(dim+1)][NP], from the warp map (coords = nullptr) or given node coordinates
// coords[c][node] of this level.
cudaError_t launch_geom_stage(const Mesh& m, const Basis1D& b, double warp_amp, const double* coords,
                              double* Jstage, cudaStream_t s);
// Geometry, stage 2: G [E][NC][NP] and wdetJ [E][NP] with mu from the formula (mu_arr = nullptr)
// or given values mu_arr[e * NP + q]. *bad (device int) is set to 1 where det J <= 0.
cudaError_t launch_geom_point(const Mesh& m, const Basis1D& b, double mu_a, double mu_b, double mu_k,
                              const double* mu_arr, const double* Jstage, double* G, double* wdetJ, int* bad,
                              cudaStream_t s);
// Gauss-point coordinates xq[c][e * NP + q] out of the stage buffer.
cudaError_t launch_extract_xq(const Mesh& m, const Basis1D& b, const double* Jstage, double* xq, cudaStream_t s);
// Node coordinates Xk[c][node] of level mesh mk from the finest level's isoparametric map
// (node coordinates X0[c][node] on mesh m0).
cudaError_t launch_level_coords(const Mesh& m0, const Basis1D& b0, const double* X0, const Mesh& mk,
                                const Basis1D& bk, double* Xk, cudaStream_t s);
// diag += diag(A) over interior nodes.
cudaError_t launch_diag(const Mesh& m, const Basis1D& b, const double* G, double* diag, cudaStream_t s);
// b += M f over interior rows.
cudaError_t launch_mass(const Mesh& m, const Basis1D& b, const double* f, double* out,
                        const double* wdetJ, cudaStream_t s);
// A[nI x nI] += interior stiffness (dense).
cudaError_t launch_elem_dense(const Mesh& m, const Basis1D& b, const double* G, double* A,
                              long long nI, cudaStream_t s);

// Element-block Jacobi (blockjac.cu). block_size_of: MI = (p-1)^d element-interior nodes per
// element (0 for p = 1). launch_elem_blocks: Kb[(e * MI + c) * MI + r] = K_e on the interior
// nodes (x fastest). launch_block_invert: each block replaced in place by its inverse; *bad
// (device int) set to 1 on a non-positive pivot. launch_block_pack: the inverses re-laid out
// into Kp (packed_block_doubles(nelem, MI) doubles, column pairs interleaved per row).
// launch_block_smooth: x_I(e) += omega * Kinv_e src_I(e) on every element's interior nodes.
// launch_mask_elem_interior: dinv = 0 at element-interior nodes.
int block_size_of(const Mesh& m);
long long packed_block_doubles(long long nelem, int MI);
cudaError_t launch_elem_blocks(const Mesh& m, const Basis1D& b, const double* G, double* Kb, cudaStream_t s);
cudaError_t launch_block_invert(double* Kb, long long nelem, int MI, int* bad, cudaStream_t s);
cudaError_t launch_block_pack(const double* Kb, double* Kp, long long nelem, int MI, cudaStream_t s);
cudaError_t launch_block_smooth(const Mesh& m, const double* Kp, const double* src, double* x, double omega,
                                cudaStream_t s);
cudaError_t launch_mask_elem_interior(double* dinv, const Mesh& m, cudaStream_t s);


}  // namespace hmg
