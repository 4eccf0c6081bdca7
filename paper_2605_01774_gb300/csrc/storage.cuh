// Population storage formats.
//
// Plain formats (FP64, FP32) keep the post-collision populations A_i(n) as they
// are.  Deviation formats keep, per node, an FP32 scale phi_s(n) and 27 16-bit
// scaled relative deviations v_i(n) from the equilibrium shape of the (uniform)
// velocity:  A_i(n) = phi_s(n) (E_i + 2^-e_i v_i(n)),  E_i = W_i P_i(u), with the
// exponents e_i = 2 + 2 m_i of lattice.cuh (W_i 2^e_i = 32/27 for all i, so v_i is the
// relative deviation (A_i/phi - E_i)/W_i times 32/27 and all 27 streams share one range).
// Encoding takes phi* = sum_i A_i, v_i = round(A_i (2^e_i/phi*) - E_i 2^e_i) (one fused
// multiply-add; exact scaling by 2^e_i commutes with the rounding), and
// phi_s = phi* / (1 + sum_i 2^-e_i v_i), so the stored node mass sum_i A_i equals phi* up
// to FP32 rounding whatever the 16-bit rounding of the v_i was.  FP16 conversion saturates
// at +-65504 and keeps NaN (a non-finite state stays visible to the reductions).
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
  // 2^-e v + c with one rounding (mixed-precision FMA: the FP16 operand enters unconverted and
  // the product with the exact power of two is exact), e.g. the decode E_i + 2^-e_i v_i
  static __device__ __forceinline__ float fma_pow2(__half v, int e, float c) {
    float r;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(r) : "h"(__half_as_ushort(v)), "h"((unsigned short)((15 - e) << 10)),
        "f"(c));
    return r;
  }
  static __device__ __forceinline__ __half from_f(float f) {
    unsigned short h;
    asm("cvt.rn.satfinite.f16.f32 %0, %1;" : "=h"(h) : "f"(f));
    return __ushort_as_half(h);
  }
};
template <>
struct Codec<__nv_bfloat16> {
  static __device__ __forceinline__ float to_f(__nv_bfloat16 h) { return __bfloat162float(h); }
  static __device__ __forceinline__ float fma_pow2(__nv_bfloat16 v, int e, float c) {
    float r;
    asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(r) : "h"(__bfloat16_as_ushort(v)),
        "h"((unsigned short)((127 - e) << 7)), "f"(c));
    return r;
  }
  static __device__ __forceinline__ __nv_bfloat16 from_f(float f) { return __float2bfloat16_rn(f); }
};

// Index of the rest population c = (0, 0, 0).
constexpr int REST = 13;

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
      return s * Codec<Elem>::fma_pow2(v, qexp_of(i), E_i);
    } else {
      return v;
    }
  }

  // Write the 27 post-collision values of node n.  Ek = E_i 2^e_i.  `mass` is sum_i a_i
  // when the caller knows it exactly (a collision conserves the node's phi); pass NaN to
  // have it summed.  Returns true where a deviation storage could not hold the node's
  // shape: when the 16-bit rounding moved the mass correction sum_i 2^-e_i v_i by 1/2 or
  // more (saturated values, or a net mass far below the populations' magnitudes), the
  // node is stored as its equilibrium shape with its mass kept (v = 0, phi_s = phi*).
  // exact (FP32 storage only): see the FP32 branch.
  static __device__ __forceinline__ bool store(Elem* __restrict__ pops, float* __restrict__ scale, int N,
                                               int n, const real (&a)[Q], const real (&Ek)[Q], real mass,
                                               bool exact = false) {
    if constexpr (dev) {
      float phi = mass;
      if (!(phi == phi)) {
        phi = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) phi += a[i];
      }
      if (fabsf(phi) > 1e-30f) {
        // the encode's rounding is compensated exactly by phi_s, so 2-ulp reciprocal suffices
        const float inv = __fdividef(1.0f, phi);
        const float ik[4] = {4.f * inv, 16.f * inv, 64.f * inv, 256.f * inv};   // 2^e / phi
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const Elem q = Codec<Elem>::from_f(fmaf(a[i], ik[nnz_of(i)], -Ek[i]));
          s = Codec<Elem>::fma_pow2(q, qexp_of(i), s);
          pops[i * N + n] = q;
        }
        if (!(fabsf(s) >= 0.5f)) {          // NaN stays on this path and stays visible
          scale[n] = phi / (1.0f + s);
          return false;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) pops[i * N + n] = Codec<Elem>::from_f(0.f);
        scale[n] = phi;
        return true;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) pops[i * N + n] = Codec<Elem>::from_f(0.f);
      scale[n] = phi;
      return false;
    } else if constexpr (std::is_same<Elem, float>::value) {
      // exact: the rounding of the node's 27 updates is put back on the rest population (c = 0,
      // so only the mass changes) and the stored sum equals the conserved phi up to the
      // rounding of that sum; otherwise that rounding acts as a small correlated source
      // (relative mass drift ~2e-8 per step on the advected plume, 7.5e-4 over 40 000 steps).
      float d = 0.f;
      if (exact && mass == mass) {
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) s += a[i];
        d = mass - s;
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) pops[i * N + n] = i == REST ? a[i] + d : a[i];
      return false;
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) pops[i * N + n] = a[i];
      return false;
    }
  }
};

}  // namespace elbm
