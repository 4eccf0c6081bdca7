// Population storage formats.
//
// Plain formats (FP64, FP32) keep the post-collision populations A_i(n) as they
// are.  Deviation formats keep, per node, an FP32 scale phi_s(n) and 27 16-bit
// relative deviations q_i(n) from the equilibrium shape of the (uniform)
// velocity:  A_i(n) = phi_s(n) (E_i + W_i q_i(n)),  E_i = W_i P_i(u).
// Encoding takes phi* = sum_i A_i, q_i = round((A_i / phi* - E_i) / W_i) and
// phi_s = phi* / (1 + sum_i W_i q_i), so the stored node mass sum_i A_i equals
// phi* up to FP32 rounding whatever the 16-bit rounding of the q_i was.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "lattice.cuh"

namespace elbm {

template <typename E>
struct Codec;
template <>
struct Codec<__half> {
  static __device__ __forceinline__ float to_f(__half h) { return __half2float(h); }
  static __device__ __forceinline__ __half from_f(float f) {
    return __float2half_rn(fminf(fmaxf(f, -65504.f), 65504.f));
  }
};
template <>
struct Codec<__nv_bfloat16> {
  static __device__ __forceinline__ float to_f(__nv_bfloat16 h) { return __bfloat162float(h); }
  static __device__ __forceinline__ __nv_bfloat16 from_f(float f) { return __float2bfloat16_rn(f); }
};

// Elem = double | float (plain) or __half | __nv_bfloat16 (deviation).
template <typename Elem>
struct Storage {
  static constexpr bool dev = !(std::is_same<Elem, double>::value || std::is_same<Elem, float>::value);
  using real = typename std::conditional<std::is_same<Elem, double>::value, double, float>::type;

  // Value of population i stored at node `src` (i is a constant after unrolling).
  static __device__ __forceinline__ real load(const Elem* __restrict__ pops, const float* __restrict__ scale,
                                              int N, int i, int src, real E_i) {
    const Elem v = __ldg(pops + (i * N + src));  // 27 N < 2^31 is checked at creation
    if constexpr (dev) {
      const float s = __ldg(scale + src);
      return s * fmaf(float(w_of(i)), Codec<Elem>::to_f(v), E_i);
    } else {
      return v;
    }
  }

  // Write the 27 post-collision values of node n.  `mass` is sum_i a_i when the caller
  // knows it exactly (a collision conserves the node's phi); pass NaN to have it summed.
  static __device__ __forceinline__ void store(Elem* __restrict__ pops, float* __restrict__ scale, int N,
                                               int n, const real (&a)[Q], const real (&E)[Q], real mass) {
    if constexpr (dev) {
      float phi = mass;
      if (!(phi == phi)) {
        phi = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) phi += a[i];
      }
      if (fabsf(phi) > 1e-30f) {
        const float inv = 1.0f / phi;
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const float r = fmaf(a[i], inv, -E[i]) * float(1.0 / w_of(i));
          const Elem q = Codec<Elem>::from_f(r);
          s = fmaf(float(w_of(i)), Codec<Elem>::to_f(q), s);
          pops[i * N + n] = q;
        }
        scale[n] = phi / (1.0f + s);
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) pops[i * N + n] = Codec<Elem>::from_f(0.f);
        scale[n] = phi;
      }
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) pops[i * N + n] = a[i];
    }
  }
};

}  // namespace elbm
