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

// The run's dynamics in the walker's precision, converted once per launch:
// the move's constants and the CV potential's coefficients.
template <typename Real>
struct MdCoef {
  int pot;
  Real c1, c2;               // dt mu, sqrt(2 mu kT dt)
  Real dwa, dwb2;            // double well: A, B^2
  Real mx, cx, my, cy;       // Mueller-Brown: the affine map of (s_0, s_1)
  Real sx, sy;               // scale * mx, scale * my
};

template <typename Real>
__device__ __forceinline__ MdCoef<Real> md_coef(const MdParams &m) {
  MdCoef<Real> k;
  k.pot = m.potential;
  k.c1 = (Real)m.c1;
  k.c2 = (Real)m.c2;
  k.dwa = (Real)m.dw_a;
  k.dwb2 = (Real)(m.dw_b * m.dw_b);
  k.mx = (Real)m.mb_map[0];
  k.cx = (Real)m.mb_map[1];
  k.my = (Real)m.mb_map[2];
  k.cy = (Real)m.mb_map[3];
  k.sx = (Real)(m.mb_scale * m.mb_map[0]);
  k.sy = (Real)(m.mb_scale * m.mb_map[2]);
  return k;
}

// One lane's Mueller-Brown term (term lane & 3 of the four), read once per
// launch so that the step loop indexes no array by lane.
template <typename Real>
struct MdTerm {
  Real A, a, b, c, x0, y0;
};

template <typename Real>
__device__ __forceinline__ MdTerm<Real> md_term(const MdParams &m, int lane) {
  const int i = lane & 3;
  return MdTerm<Real>{(Real)m.mb_A[i], (Real)m.mb_a[i], (Real)m.mb_b[i], (Real)m.mb_c[i], (Real)m.mb_x0[i],
                      (Real)m.mb_y0[i]};
}

// dU/ds_k of the run's CV potential (abp.h: ABP_POT_*) by the warp: lane i <
// 4 forms the i-th Mueller-Brown term (its coefficients in mt), the four are
// summed by two lane exchanges ((t0 + t1) + (t2 + t3)); lane 0 returns the
// gradient.
template <typename Real>
__device__ __forceinline__ void md_potential_grad_warp(const MdCoef<Real> &k, const MdTerm<Real> &mt, const Real *s,
                                                       int lane, Real *dU) {
  dU[0] = dU[1] = dU[2] = 0;
  if (k.pot == ABP_POT_DOUBLE_WELL) {
    dU[0] = (Real)4 * k.dwa * s[0] * (s[0] * s[0] - k.dwb2);
  } else if (k.pot == ABP_POT_MULLER_BROWN) {
    Real gx = 0, gy = 0;
    if (lane < 4) {
      const Real X = k.mx * s[0] + k.cx, Y = k.my * s[1] + k.cy;
      const Real xp = X - mt.x0, yp = Y - mt.y0;
      const Real e = mt.A * exp(mt.a * xp * xp + mt.b * xp * yp + mt.c * yp * yp);
      gx = e * ((Real)2 * mt.a * xp + mt.b * yp);
      gy = e * (mt.b * xp + (Real)2 * mt.c * yp);
    }
    gx += __shfl_xor_sync(0xffffffffu, gx, 1);
    gy += __shfl_xor_sync(0xffffffffu, gy, 1);
    gx += __shfl_xor_sync(0xffffffffu, gx, 2);
    gy += __shfl_xor_sync(0xffffffffu, gy, 2);
    dU[0] = k.sx * gx;
    dU[1] = k.sy * gy;
  }
}

}  // namespace abp
