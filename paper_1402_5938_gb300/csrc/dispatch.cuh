// Runtime-to-compile-time dispatch helpers for the element kernels.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "element.cuh"

namespace hmg {

template <typename F>
cudaError_t dispatch_n(int n, F&& f) {
  switch (n) {
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 7: return f(std::integral_constant<int, 7>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 9: return f(std::integral_constant<int, 9>{});
    case 10: return f(std::integral_constant<int, 10>{});
    case 11: return f(std::integral_constant<int, 11>{});
    case 12: return f(std::integral_constant<int, 12>{});
    case 13: return f(std::integral_constant<int, 13>{});
    case 14: return f(std::integral_constant<int, 14>{});
    case 15: return f(std::integral_constant<int, 15>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 17: return f(std::integral_constant<int, 17>{});
    default: return cudaErrorInvalidValue;
  }
}

template <int N, typename T>
Tab<N, T> make_tab(const Basis1D& b) {
  Tab<N, T> t;
  for (int i = 0; i < N * N; ++i) {
    t.B[i] = (T)b.B[i];
    t.D[i] = (T)b.D[i];
  }
  return t;
}

template <int N>
GeoTab<N> make_geotab(const Basis1D& b) {
  GeoTab<N> t;
  for (int i = 0; i < N * N; ++i) {
    t.B[i] = b.B[i];
    t.D[i] = b.D[i];
    t.Bd[i] = b.Bd[i];
    t.BB[i] = b.B[i] * b.B[i];
    t.BD[i] = b.B[i] * b.Bd[i];
    t.DD[i] = b.Bd[i] * b.Bd[i];
  }
  for (int i = 0; i < N; ++i) {
    t.r[i] = b.r[i];
    t.w[i] = b.w[i];
  }
  return t;
}

// Opt a kernel into more than 48 KB of dynamic shared memory (once per kernel and device).
cudaError_t ensure_smem_ptr(const void* kernel, size_t bytes);
template <typename K>
cudaError_t ensure_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return ensure_smem_ptr((const void*)kernel, bytes);
}

// Elements per block: fill about 64 KB of shared memory, at least one element.
inline int epb_for(size_t per_elem_bytes) {
  size_t e = (64 * 1024) / per_elem_bytes;
  if (e < 1) e = 1;
  if (e > 64) e = 64;
  return (int)e;
}

}  // namespace hmg
