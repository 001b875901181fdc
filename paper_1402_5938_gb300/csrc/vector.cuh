// Level-vector kernels: deterministic reductions, smoother and PCG updates, 1D transfer
// passes, the dense coarsest solve, and the Arnoldi helpers.
#pragma once

#include "common.cuh"

namespace hmg {

// Scalars kept on the device (no host round trip inside an iteration).
enum Scalar : int {
  S_RHO = 0,    // (z, r) of PCG
  S_PH = 1,     // (p, A p)
  S_RR = 2,     // ||r||^2
  S_BETA = 3,   // PCG beta
  S_TMP = 4,    // scratch scalar (Arnoldi h_ij, norms)
  S_RR0 = 5,    // ||r_0||^2
  S_RTOL = 6,   // relative tolerance of a graph solve
  S_LRR0 = 8,   // ||r_0||^2 of a lockstep (batched) solve
  S_LRR = 9,    // ||r||^2 of a lockstep solve (copied to the host with S_LRR0)
  S_COUNT = 10
};

// Device-side solve control of a graph solve: ctrl[0] iteration, ctrl[1] status, ctrl[2] maxit,
// ctrl[3] capacity of the residual-history array.
enum SolveStatus : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAXIT = 2, ST_NAN = 3 };

enum FinishOp : int { FIN_STORE = 0, FIN_SQRT = 1, FIN_RHO_BETA = 2, FIN_NEG_RATIO = 3 };

constexpr int kRedBlocks = 1216;  // fixed partial count (8 x 152 SMs); fixed => deterministic sums

// Axis transfer: one 1D CSR matrix (rows = output indices along the axis).
struct Axis1D {
  int n_out, n_in;
  int* rowptr;       // device, n_out + 1
  int* col;          // device, nnz
  double* val;       // device, nnz
  float* val32;      // device, nnz
};

// One output point t of a 1D transfer pass along `axis` (Sec. 2.2: P and R = P^T act as
// Kronecker products of 1D factors, applied one axis at a time). The output has extents
// o0 x o1 x o2 (x fastest); the input has n_in points along `axis` and the output's extents on
// the other two. mask_in skips input points on the box boundary (Dirichlet nodes), mask_out
// zeroes output points on it (with acc: leaves them). 32-bit indexing: every level vector and
// pass intermediate has fewer than 2^31 entries (meshes are validated below that). The point
// decode is two 32-bit divisions, the input base and the boundary tests of the two other axes
// are taken once per output, and the row's entries are summed in CSR order.
template <typename T, typename V>
__device__ __forceinline__ void axis_point(const T* __restrict__ in, T* __restrict__ out, unsigned t,
                                           unsigned o0, unsigned o1, unsigned o2, int axis, int n_in,
                                           const int* __restrict__ rowptr, const int* __restrict__ col,
                                           const V* __restrict__ val, int mask_in, int mask_out, int acc) {
  const unsigned q = t / o0, i0 = t - q * o0;
  const unsigned i2 = q / o1, i1 = q - i2 * o1;
  const bool b0 = o0 > 1 && (i0 == 0 || i0 == o0 - 1);
  const bool b1 = o1 > 1 && (i1 == 0 || i1 == o1 - 1);
  const bool b2 = o2 > 1 && (i2 == 0 || i2 == o2 - 1);
  const bool obd = mask_out && (b0 || b1 || b2);
  unsigned row, base, stride;
  bool other_bd;
  if (axis == 0) {
    row = i0, base = (unsigned)n_in * (i1 + o1 * i2), stride = 1, other_bd = b1 || b2;
  } else if (axis == 1) {
    row = i1, base = i0 + o0 * (unsigned)n_in * i2, stride = o0, other_bd = b0 || b2;
  } else {
    row = i2, base = i0 + o0 * i1, stride = o0 * o1, other_bd = b0 || b1;
  }
  T s = T(0);
  if (!obd && !(mask_in && other_bd)) {
    const int k1 = rowptr[row + 1];
    for (int k = rowptr[row]; k < k1; ++k) {
      const int c = col[k];
      if (mask_in && n_in > 1 && (c == 0 || c == n_in - 1)) continue;
      s = fma((T)val[k], in[base + (unsigned)c * stride], s);
    }
  }
  if (acc) {
    if (!obd) out[t] += s;
  } else {
    out[t] = s;
  }
}

// reductions over n entries: red_blocks(n) partials, then finish into S (pass the same n)
int red_blocks(long long n);
cudaError_t dot_partial(const double* x, const double* y, long long n, double* partial, cudaStream_t s);
cudaError_t dot_partial_f32(const float* x, const float* y, long long n, double* partial, cudaStream_t s);
cudaError_t finish(const double* partial, long long n, double* S, int op, int idx, int aux, double* host_copy,
                   cudaStream_t s);

// PCG: alpha = S_RHO / S_PH; u += alpha p; r -= alpha h; partial <- ||r||^2
cudaError_t pcg_update(double* u, double* r, const double* p, const double* h, long long n,
                       const double* S, double* partial, cudaStream_t s);
// p = z + S_BETA * p
cudaError_t pcg_direction(double* p, const double* z, long long n, const double* S, cudaStream_t s);

// smoother updates (T = double or float); `r` (nullable) / reset_r also write r = b for the next
// residual apply
template <typename T>
cudaError_t jacobi_first(T* x, const T* b, const T* dinv, long long n, T omega, cudaStream_t s, T* r = nullptr);
template <typename T>
cudaError_t jacobi_step(T* x, T* r, const T* b, const T* dinv, long long n, T omega, int reset_r,
                        cudaStream_t s);
template <typename T>
cudaError_t cheb_first(T* x, T* d, const T* b, const T* dinv, long long n, T inv_theta, cudaStream_t s,
                       T* r = nullptr);
template <typename T>
cudaError_t cheb_step(T* x, T* d, T* r, const T* b, const T* dinv, long long n, T c1, T c2, int reset_r,
                      cudaStream_t s);

cudaError_t dinv_from_diag(const double* diag, double* dinv, long long n, cudaStream_t s);
cudaError_t mask_boundary(double* v, const Mesh& m, cudaStream_t s);
cudaError_t copy_masked(double* dst, const double* src, const Mesh& m, cudaStream_t s);
cudaError_t to_f32(float* dst, const double* src, long long n, cudaStream_t s);
cudaError_t to_f64(double* dst, const float* src, long long n, cudaStream_t s);

// Arnoldi helpers
cudaError_t start_vector(double* v, const Mesh& m, unsigned long long seed, cudaStream_t s);
cudaError_t scale_by(double* w, const double* dinv, long long n, cudaStream_t s);
// l1 row norms by probing: v = indicator of the interior nodes in one color class (axis indices
// congruent to (c0, c1, c2) mod period), and acc += |y| after y = A v.
cudaError_t color_indicator(double* v, const Mesh& m, int period, int c0, int c1, int c2, cudaStream_t s);
cudaError_t accum_abs(double* acc, const double* y, long long n, cudaStream_t s);
// One classical Gram-Schmidt pass against the cnt vectors V_i = V + i * ldv: c = V^T w,
// H[i * ldh] += c[i], w -= V c (partial: cnt * red_blocks(n) doubles; c: cnt doubles).
cudaError_t project_out(double* w, const double* V, long long ldv, int cnt, long long n, double* partial,
                        double* c, double* H, int ldh, cudaStream_t s);
cudaError_t axpy_dev(double* y, const double* x, long long n, const double* coef, double sign, cudaStream_t s);
cudaError_t div_dev(double* y, const double* x, long long n, const double* den, cudaStream_t s);
cudaError_t copy_scalar(double* dst, const double* src, cudaStream_t s);
cudaError_t axpy(double* y, const double* x, long long n, double a, cudaStream_t s);
// xyz[c*N + g] = physical coordinate c of node g (warp of the reference GLL grid)
cudaError_t node_coords(double* xyz, const Mesh& m, const double* gll, double warp_amp, cudaStream_t s);

// out (=, or += if accumulate) M_axis in, for a 3D array with output dims od[3]; input dims
// equal od except along `axis` (n_in). mask_in: treat input nodes on the input grid's
// boundary as zero; mask_out: write zero on output boundary nodes (no accumulation).
template <typename T>
cudaError_t axis_pass(const T* in, T* out, const long long od[3], int axis, const Axis1D& M, int mask_in,
                      int mask_out, int accumulate, cudaStream_t s);

// Dense coarsest level: Gauss-Jordan inverse in place (SPD, no pivoting), and the solve
// x[gmap[i]] = sum_j Ainv[i][j] b[gmap[j]].
// The inverse by 32-wide panels (block Gauss-Jordan: invert the pivot block, scale its rows,
// rank-32 update of the rest by an FP64 GEMM, then the pivot columns and rows): n/32 panels of 7
// operations instead of 2n launches. work: blocked_gj_work_doubles(n) doubles; *bad (device int)
// is set when a pivot block has a non-positive pivot.
size_t blocked_gj_work_doubles(long long n);
cudaError_t blocked_gauss_jordan_inverse(double* A, long long n, double* work, int* bad, cudaStream_t s);
cudaError_t coarse_solve(const double* Ainv, const double* b, double* x, const long long* gmap,
                         long long nI, cudaStream_t s);
cudaError_t coarse_solve_f32(const double* Ainv, const float* b, float* x, const long long* gmap,
                             long long nI, cudaStream_t s);

// one block waits (bounded, `polls` polls) on a barrier nothing completes; *out_dev = 1 if it gave up
cudaError_t bounded_wait_probe(unsigned polls, int* out_dev, cudaStream_t s);

// graph-solve control kernels (single thread): parameters, start check, per-iteration check.
// The checks set the WHILE condition `hw` (and the IF condition `hi` if has_if) to "continue".
cudaError_t set_solve_params(double* S, int* ctrl, double rtol, int maxit, int cap, cudaStream_t s);
cudaError_t start_check(const double* S, int* ctrl, double* hist, cudaGraphConditionalHandle hw, cudaStream_t s);
cudaError_t step_check(const double* S, int* ctrl, double* hist, cudaGraphConditionalHandle hw,
                       cudaGraphConditionalHandle hi, int has_if, cudaStream_t s);

}  // namespace hmg
