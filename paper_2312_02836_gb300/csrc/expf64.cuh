// expf64.cuh -- FP64 exp for the rate fits, written from Tang's table-driven
// method (P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989).
//
//   N = round(x * 32/ln2), j = N mod 32, M = (N - j)/32
//   r = x - N (ln2/32)          (two-part constant, each part applied by FMA)
//   p = r + r^2/2 + ... + r^6/720   (|r| <= ln2/64: truncation < 2e-18)
//   exp(x) = 2^M * (S_j + S_j p),   S_j = 2^(j/32) as a double-double
//
// About 12 FP64 instructions against ~20 DFMA-equivalents for the general
// library exp measured on GB300; the FP64 pipe is this kernel's bottleneck.
// Results outside |x| <= 700 (overflow, underflow, subnormals, NaN) are
// handed to the library exp.  Error bound: below 0.6 ulp (tested against
// the CUDA exp on the GPU and against mpmath on the host).
#pragma once
#ifndef __CUDACC_RTC__  // the run-time compiler has no system headers
#include <math.h>
#include <stdint.h>
#include <string.h>
#endif

#ifndef NB_HD
#define NB_HD __device__
#endif

namespace nb {

// S_j = 2^(j/32) = lead + trail, j = 0..31 (mpmath, 200-bit; printed by
// exp2_table.py beside this header)
#define NB_EXP2_TABLE                                                     \
  0x1.0000000000000p+0, 0x0.0p+0, 0x1.059b0d3158574p+0, 0x1.d73e2a475b465p-55, \
  0x1.0b5586cf9890fp+0, 0x1.8a62e4adc610bp-54, 0x1.11301d0125b51p+0, -0x1.6c51039449b3ap-54, \
  0x1.172b83c7d517bp+0, -0x1.19041b9d78a76p-55, 0x1.1d4873168b9aap+0, 0x1.e016e00a2643cp-54, \
  0x1.2387a6e756238p+0, 0x1.9b07eb6c70573p-54, 0x1.29e9df51fdee1p+0, 0x1.612e8afad1255p-55, \
  0x1.306fe0a31b715p+0, 0x1.6f46ad23182e4p-55, 0x1.371a7373aa9cbp+0, -0x1.63aeabf42eae2p-54, \
  0x1.3dea64c123422p+0, 0x1.ada0911f09ebcp-55, 0x1.44e086061892dp+0, 0x1.89b7a04ef80d0p-59, \
  0x1.4bfdad5362a27p+0, 0x1.d4397afec42e2p-56, 0x1.5342b569d4f82p+0, -0x1.07abe1db13cadp-55, \
  0x1.5ab07dd485429p+0, 0x1.6324c054647adp-54, 0x1.6247eb03a5585p+0, -0x1.383c17e40b497p-54, \
  0x1.6a09e667f3bcdp+0, -0x1.bdd3413b26456p-54, 0x1.71f75e8ec5f74p+0, -0x1.16e4786887a99p-55, \
  0x1.7a11473eb0187p+0, -0x1.41577ee04992fp-55, 0x1.82589994cce13p+0, -0x1.d4c1dd41532d8p-54, \
  0x1.8ace5422aa0dbp+0, 0x1.6e9f156864b27p-54, 0x1.93737b0cdc5e5p+0, -0x1.75fc781b57ebcp-57, \
  0x1.9c49182a3f090p+0, 0x1.c7c46b071f2bep-56, 0x1.a5503b23e255dp+0, -0x1.d2f6edb8d41e1p-54, \
  0x1.ae89f995ad3adp+0, 0x1.7a1cd345dcc81p-54, 0x1.b7f76f2fb5e47p+0, -0x1.5584f7e54ac3bp-56, \
  0x1.c199bdd85529cp+0, 0x1.11065895048ddp-55, 0x1.cb720dcef9069p+0, 0x1.503cbd1e949dbp-56, \
  0x1.d5818dcfba487p+0, 0x1.2ed02d75b3707p-55, 0x1.dfc97337b9b5fp+0, -0x1.1a5cd4f184b5cp-54, \
  0x1.ea4afa2a490dap+0, -0x1.e9c23179c2893p-54, 0x1.f50765b6e4540p+0, 0x1.9d3e12dd8a18bp-54

#ifdef __CUDACC__
__device__ const double g_exp2_table[64] = {NB_EXP2_TABLE};
#endif
#ifndef __CUDACC_RTC__
static const double h_exp2_table[64] = {NB_EXP2_TABLE};
#endif

NB_HD __forceinline__ double exp_tang(double x) {
#ifdef __CUDA_ARCH__
  const double* tab = g_exp2_table;
#else
  const double* tab = h_exp2_table;
#endif
  long long xb;
#ifdef __CUDA_ARCH__
  xb = __double_as_longlong(x);
#else
  memcpy(&xb, &x, sizeof(xb));
#endif
  // |x| <= 700 (and not NaN), decided on the bits: 0x4085e00000000000 = 700.0
  if ((xb & 0x7fffffffffffffffLL) > 0x4085e00000000000LL) return exp(x);
  const double kInvL = 0x1.71547652b82fep+5;   // 32 / ln 2
  const double kL1 = 0x1.62e42fefa39efp-6;     // ln2/32, leading part
  const double kL2 = 0x1.abc9e3b39803fp-61;    // ln2/32 - kL1
  const double kShift = 0x1.8p52;              // rounds to an integer
  const double t = fma(x, kInvL, kShift);
  const double Nd = t - kShift;
  long long tb;
#ifdef __CUDA_ARCH__
  tb = __double_as_longlong(t);
#else
  memcpy(&tb, &t, sizeof(tb));
#endif
  const int N = (int)(tb & 0xffffffffLL);        // low bits hold round(x*32/ln2)
  const int j = N & 31;
  const int M = (N - j) >> 5;
  double r = fma(-Nd, kL1, x);
  r = fma(-Nd, kL2, r);
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(q, r * r, r);
#ifdef __CUDA_ARCH__
  const double lead = __ldg(tab + 2 * j), trail = __ldg(tab + 2 * j + 1);
#else
  const double lead = tab[2 * j], trail = tab[2 * j + 1];
#endif
  const double v = lead + fma(lead, p, trail);   // in [1, 2)
  long long vb;
#ifdef __CUDA_ARCH__
  vb = __double_as_longlong(v) + ((long long)M << 52);
  return __longlong_as_double(vb);
#else
  memcpy(&vb, &v, sizeof(vb));
  vb += (long long)M << 52;
  double out;
  memcpy(&out, &vb, sizeof(out));
  return out;
#endif
}

}  // namespace nb
