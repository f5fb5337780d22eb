// RK epilogue of the FP64 gather-scatter kernels (single problem and batch):
// out[o] = alpha_k[o][nsh] a + sum_m beta[o][m] src[m] for the assembled value
// a of a node shared by 2^nsh elements (Epi in sem_internal.h).
#pragma once
#include <cuda_runtime.h>

#include "sem_internal.h"

namespace semk {

// FP64 work per unique node: (contributions - 1) adds, then per output one
// multiply (none when alpha is 1) and one fused multiply-add per source with a
// nonzero coefficient (epi_output below).  The FP64 pipe of GB300 issues
// two lanes per SM per clock, so everything else (the non-finite test on the
// exponent bits, the choice of contributions, the index arithmetic) stays on the
// integer pipes.
__device__ __forceinline__ bool nonfinite_bits(double v) {
    return (__double2hiint(v) & 0x7ff00000) == 0x7ff00000;
}

// alpha_k[o][nsh] of a kernel-parameter table, picked with selects on the four
// statically addressed entries: an indexed parameter load would be a
// dependent constant-cache access on the path of every thread.
template <typename A>
__device__ __forceinline__ A pick4(const A (&t)[4], int k) {
    const A lo = k & 1 ? t[1] : t[0];
    const A hi = k & 1 ? t[3] : t[2];
    return k & 2 ? hi : lo;
}

// Host side: fold the 1/k multiplicity of F and J into alpha_k and build the
// per-output keys of epi_output.
inline void epi_prepare(Epi& ep, int scale_mult) {
    for (int o = 0; o < 3; ++o) {
        for (int k = 0; k < 4; ++k) ep.alpha_k[o][k] = scale_mult ? ep.alpha[o] / (double)(1 << k) : ep.alpha[o];
        unsigned key = ep.alpha[o] == 1.0 ? (scale_mult ? 32u : 16u) : 0u;
        for (int m = 0; m < ep.nsrc && m < 4; ++m)
            if (ep.beta[o][m] != 0.0) key |= 1u << m;
        ep.key[o] = key;
    }
}

// a * 2^-k (k = 0..3) without an FP64 instruction: the exponent field is lowered with
// integer arithmetic, which is exact.  Zeros, subnormal results, infinities and NaNs
// (rare) take the multiply, which gives the same value.
__device__ __forceinline__ double epi_pow2_down(double a, int k) {
    const long long b = __double_as_longlong(a);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex > k && ex != 0x7ff) return __longlong_as_double(b - ((long long)k << 52));
    return a * (k == 0 ? 1.0 : (k == 1 ? 0.5 : (k == 2 ? 0.25 : 0.125)));
}

// The terms of one RK-epilogue output are fixed at compile time by KEY: bit m
// when source m enters (beta != 0), bit 4 when alpha_k == 1 (no 1/k scaling),
// bit 5 when alpha == 1 with the 1/k scaling (alpha_k = 2^-nsh, applied to the
// exponent on the integer pipe); v = alpha_k a + sum over the set bits of
// beta_m src_m, in source order.  The
// host builds the key per launch, so the switch below is a branch that every
// thread takes the same way, and a skipped term issues no instruction: a
// predicated-off FP64 instruction would still occupy the FP64 pipe.  Leaving
// out a zero term or a unit multiply does not change the result.
#define SEMK_KEY_CASES(X)                                                                    \
    X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15)   \
    X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29)     \
    X(30) X(31) X(32) X(33) X(34) X(35) X(36) X(37) X(38) X(39) X(40) X(41) X(42) X(43)     \
    X(44) X(45) X(46) X(47)

template <int R, int NSRC, unsigned KEY>
__device__ __forceinline__ void epi_terms(double (&v)[R], const double (&a)[R], const double (&sum)[R],
                                          const double (&b)[4], const double (&sv)[R][NSRC > 0 ? NSRC : 1],
                                          const int (&nsh)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
        double x = (KEY & 16u) ? sum[r] : ((KEY & 32u) ? epi_pow2_down(sum[r], nsh[r]) : a[r] * sum[r]);
#pragma unroll
        for (int m = 0; m < NSRC; ++m)
            if ((KEY >> m) & 1u) x = fma(b[m], sv[r][m], x);
        v[r] = x;
    }
}

template <int R, int NSRC>
__device__ __forceinline__ void epi_output(unsigned key, double (&v)[R], const double (&a)[R],
                                           const double (&sum)[R], const double (&b)[4],
                                           const double (&sv)[R][NSRC > 0 ? NSRC : 1], const int (&nsh)[R]) {
    constexpr unsigned FULL = (1u << NSRC) - 1u;
    switch (key) {
#define SEMK_EPI_CASE(K)                                                     \
    case K:                                                                  \
        if constexpr ((K & 15u) <= FULL) {                                   \
            epi_terms<R, NSRC, K>(v, a, sum, b, sv, nsh);                    \
            return;                                                          \
        }                                                                    \
        break;
        SEMK_KEY_CASES(SEMK_EPI_CASE)
#undef SEMK_EPI_CASE
    }
    epi_terms<R, NSRC, FULL>(v, a, sum, b, sv, nsh);   // not reached: keys come from the sources
}

}  // namespace semk
