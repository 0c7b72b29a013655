// abp_md.cuh -- the noise and the CV potential of the closed-loop form
// (abp_md_run), shared by its kernels (abp_md.cu, the phased form's move in
// abp_big.cu).
#pragma once

#include <cuda_runtime.h>

#include "abp_internal.cuh"

namespace abp {

// Philox-4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, SC'11): a round
// multiplies counter words 0 and 2 by the round multipliers and forms
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
// advances by the Weyl increments before every round but the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Three standard normals of one atom at one step (the counter and key of
// abp.h; Box-Muller on (j + 1/2) 2^-24, j the word's top 24 bits).
__device__ __forceinline__ void md_normals(unsigned long long seed, unsigned stream, long long step, int atom,
                                           float *n) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)atom, (unsigned)step, (unsigned)((unsigned long long)step >> 32),
                                           stream),
                                make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const float u0 = ((float)(r.x >> 8) + 0.5f) * 5.9604644775390625e-8f;
  const float u1 = ((float)(r.y >> 8) + 0.5f) * 5.9604644775390625e-8f;
  const float u2 = ((float)(r.z >> 8) + 0.5f) * 5.9604644775390625e-8f;
  const float u3 = ((float)(r.w >> 8) + 0.5f) * 5.9604644775390625e-8f;
  const float r0 = sqrtf(-2.f * logf(u0)), r2 = sqrtf(-2.f * logf(u2));
  float sn, cs;
  sincospif(2.f * u1, &sn, &cs);
  n[0] = r0 * cs;
  n[1] = r0 * sn;
  n[2] = r2 * cospif(2.f * u3);
}
__device__ __forceinline__ void md_normals(unsigned long long seed, unsigned stream, long long step, int atom,
                                           double *n) {
  const uint4 r = philox4x32_10(make_uint4((unsigned)atom, (unsigned)step, (unsigned)((unsigned long long)step >> 32),
                                           stream),
                                make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const double u0 = ((double)(r.x >> 8) + 0.5) * 5.9604644775390625e-8;
  const double u1 = ((double)(r.y >> 8) + 0.5) * 5.9604644775390625e-8;
  const double u2 = ((double)(r.z >> 8) + 0.5) * 5.9604644775390625e-8;
  const double u3 = ((double)(r.w >> 8) + 0.5) * 5.9604644775390625e-8;
  const double r0 = sqrt(-2.0 * log(u0)), r2 = sqrt(-2.0 * log(u2));
  double sn, cs;
  sincospi(2.0 * u1, &sn, &cs);
  n[0] = r0 * cs;
  n[1] = r0 * sn;
  n[2] = r2 * cospi(2.0 * u3);
}

// dU/ds_k of the run's CV potential (abp.h: ABP_POT_*).
template <typename Real>
__device__ __forceinline__ void md_potential_grad(const MdParams &m, const Real *s, Real *dU) {
  dU[0] = dU[1] = dU[2] = 0;
  if (m.potential == ABP_POT_DOUBLE_WELL) {
    const Real b = (Real)m.dw_b, q = s[0] * s[0] - b * b;
    dU[0] = (Real)4 * (Real)m.dw_a * s[0] * q;
  } else if (m.potential == ABP_POT_MULLER_BROWN) {
    const Real X = (Real)m.mb_map[0] * s[0] + (Real)m.mb_map[1];
    const Real Y = (Real)m.mb_map[2] * s[1] + (Real)m.mb_map[3];
    Real dX = 0, dY = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const Real xp = X - (Real)m.mb_x0[i], yp = Y - (Real)m.mb_y0[i];
      const Real a = (Real)m.mb_a[i], b = (Real)m.mb_b[i], c = (Real)m.mb_c[i];
      const Real e = (Real)m.mb_A[i] * exp(a * xp * xp + b * xp * yp + c * yp * yp);
      dX += e * ((Real)2 * a * xp + b * yp);
      dY += e * (b * xp + (Real)2 * c * yp);
    }
    dU[0] = (Real)m.mb_scale * (Real)m.mb_map[0] * dX;
    dU[1] = (Real)m.mb_scale * (Real)m.mb_map[2] * dY;
  }
}

}  // namespace abp
