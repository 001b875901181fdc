// Host launchers of the element kernels, dispatched from the runtime order p to the
// compile-time node count N = p + 1 (2..17).
#pragma once

#include "common.cuh"

namespace hmg {

// y += alpha * A x (FP64 or FP32 data; G in the same precision). Both kernels stage G with
// bulk TMA copies (FP64: when the slab fits in shared memory) and need G allocated with >= 16
// bytes of tail padding; a timed-out wait sets *err (device int) to a nonzero code.
// `variant` selects the block shape (FP64: 0..3, 3 = TMA-staged G; FP32: 0..2 tile sizes); setup
// picks it per level by timing (autotuning).
constexpr int kApply64Variants = 4;
constexpr int kApply32Variants = 3;
cudaError_t launch_apply_f64(const Mesh& m, const Basis1D& b, const double* x, double* y,
                             const double* G, double alpha, int* err, cudaStream_t s, int variant = 0);
cudaError_t launch_apply_f32(const Mesh& m, const Basis1D& b, const float* x, float* y,
                             const float* G, float alpha, int* err, cudaStream_t s, int variant = 0);

// Geometry: stage buffer J [E][dim*(dim+1)][NP], then G [E][NC][NP] and wdetJ [E][NP].
// *bad (device int) is set to 1 where det J <= 0.
cudaError_t launch_geometry(const Mesh& m, const Basis1D& b, double warp_amp, double mu_a,
                            double mu_b, double mu_k, double* Jstage, double* G, double* wdetJ,
                            int* bad, cudaStream_t s);
// diag += diag(A) over interior nodes.
cudaError_t launch_diag(const Mesh& m, const Basis1D& b, const double* G, double* diag, cudaStream_t s);
// b += M f over interior rows.
cudaError_t launch_mass(const Mesh& m, const Basis1D& b, const double* f, double* out,
                        const double* wdetJ, cudaStream_t s);
// A[nI x nI] += interior stiffness (dense).
cudaError_t launch_elem_dense(const Mesh& m, const Basis1D& b, const double* G, double* A,
                              long long nI, cudaStream_t s);


}  // namespace hmg
