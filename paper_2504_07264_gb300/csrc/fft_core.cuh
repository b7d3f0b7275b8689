// fft_core.cuh -- register-level building blocks of the planar FP32 DFT.
//
// The transform of Eq. (1) is computed in the split form of Eq. (3): real and
// imaginary parts live in separate float registers and separate planar
// arrays, and every complex product is written out on (re, im) pairs, i.e.
// the 2x2 rotation blocks omega^(i,q) of Section III (definitions under
// Eq. (6)) applied to a pair.
//
// Organisation on the GPU.  Eq. (6) is the radix-2 Cooley-Tukey factorisation
// of E_2N.  Its stages can be regrouped: a DFT of size N = R * Q splits into R-point
// DFTs over the top digit of n, a twiddle rotation by W_N^{nl * d}, and Q-point
// DFTs over the remaining digits (the same butterfly W(i) and rotation D(i)
// factors of Eq. (6), applied in decimation-in-frequency order, cf. Eq. (9)).
// Each "step" below is one such regrouping: every thread runs small DFTs
// entirely in registers (split-radix DIF butterflies with compile-time rotation
// constants), then rotates by per-plan twiddle tables, then exchanges data
// through shared memory for the next step.  The final step writes natural
// order, so the permutation S of Eq. (6) never materialises: it is absorbed
// into register numbering (compile-time) and the exchange addressing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdft {

// W_64^q = exp(-j 2 pi q / 64) = c[q] + j s[q]  (s[q] = -sin(2 pi q / 64)),
// computed in float64 and rounded once (see twiddle.cu).  Passed by value as
// a kernel parameter so compile-time indexed reads become constant-bank
// operands.  Every register DFT of size L <= 64 takes W_L^q = W_64^{q*64/L}.
struct W64 {
    float c[64];
    float s[64];
};

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

__host__ __device__ constexpr int brevc(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// (r + j i) <- (r + j i) * W_L^q, or * conj(W_L^q) for the adjoint, for a
// compile-time (q, L) with 0 <= q < L/2, L <= 64.  This is the 2x2 block
// omega^(i,q) (Section III) acting on the pair (r, i); q = 0, L/4 (a quarter
// turn), L/8 and 3L/8 (eighth turns) are written out so that they cost no
// general multiply.
template <bool ADJ>
__device__ __forceinline__ void rot_const(float& r, float& i, const int q, const int L,
                                          const W64& w) {
    if (q == 0) return;
    if (4 * q == L) {                      // W = -j (forward), +j (adjoint)
        const float a = r;
        if (!ADJ) { r = i; i = -a; } else { r = -i; i = a; }
        return;
    }
    const float h = 0.70710678118654752440f;
    if (8 * q == L) {                      // W = (1 - j)/sqrt2, adjoint (1 + j)/sqrt2
        const float a = r, b = i;
        if (!ADJ) { r = (a + b) * h; i = (b - a) * h; }
        else      { r = (a - b) * h; i = (a + b) * h; }
        return;
    }
    if (8 * q == 3 * L) {                  // W = -(1 + j)/sqrt2, adjoint (-1 + j)/sqrt2
        const float a = r, b = i;
        if (!ADJ) { r = (b - a) * h; i = -(a + b) * h; }
        else      { r = -(a + b) * h; i = (a - b) * h; }
        return;
    }
    const int idx = q * (64 / L);
    const float c = w.c[idx];
    const float s = ADJ ? -w.s[idx] : w.s[idx];
    const float nr = r * c - i * s;
    const float ni = r * s + i * c;
    r = nr;
    i = ni;
}

// (r + j i) <- (r + j i) * (c + j s), or * (c - j s) for the adjoint.
template <bool ADJ>
__device__ __forceinline__ void rot(float& r, float& i, const float2 w) {
    const float c = w.x;
    const float s = ADJ ? -w.y : w.y;
    const float nr = r * c - i * s;
    const float ni = r * s + i * c;
    r = nr;
    i = ni;
}

// (r + j i) <- (r + j i) * W_L^q (conjugate for the adjoint) for a
// compile-time q anywhere on the circle, 0 <= q < L <= 64: the quarter turns
// and the odd eighths written out, the rest from the W_64 constants.
template <bool ADJ>
__device__ __forceinline__ void rot_any(float& r, float& i, const int q, const int L,
                                        const W64& w) {
    if (q == 0) return;
    if (2 * q == L) {                      // -1
        r = -r;
        i = -i;
        return;
    }
    if (4 * q == L || 4 * q == 3 * L) {    // -j, or +j for three quarters (conjugated: adjoint)
        const bool minus_j = (4 * q == L) != ADJ;
        const float a = r;
        if (minus_j) { r = i; i = -a; } else { r = -i; i = a; }
        return;
    }
    if ((8 * q) % L == 0) {                // odd eighths: (+-1 +- j)/sqrt2
        const float h = 0.70710678118654752440f;
        const int m = 8 * q / L;           // W_8^m, m = 1, 3, 5, 7
        const float c = (m == 1 || m == 7) ? h : -h;
        const float sf = (m == 1 || m == 3) ? -h : h;
        const float sv = ADJ ? -sf : sf;
        const float a = r, b = i;
        r = a * c - b * sv;
        i = a * sv + b * c;
        return;
    }
    const int idx = q * (64 / L);
    const float c = w.c[idx];
    const float sv = ADJ ? -w.s[idx] : w.s[idx];
    const float nr = r * c - i * sv;
    const float ni = r * sv + i * c;
    r = nr;
    i = ni;
}

// In-register L-point DFT of re/im[off .. off+L-1] (natural input order) by
// split-radix decimation in frequency: with t1 = x_n - x_{n+L/2} and
// t2 = x_{n+L/4} - x_{n+3L/4} (n < L/4),
//   first half     x_n + x_{n+L/2}            -> the L/2-point DFT: X[2k]
//   third quarter  (t1 - j t2) W_L^n          -> L/4-point DFT:     X[4k+1]
//   fourth quarter (t1 + j t2) W_L^{3n}       -> L/4-point DFT:     X[4k+3]
// (+j and -j exchanged, rotations conjugated, for the adjoint).  These are the
// radix-2 factors W(i) and D(i) of Eq. (6) regrouped so that two stages share
// one rotation; bin k lands in register off + brevc(k, log2 L), the order the
// radix-2 form gives.
template <int L, bool ADJ, int E>
__device__ __forceinline__ void dft_split_radix(float (&re)[E], float (&im)[E], const int off,
                                                const W64& w) {
    if constexpr (L == 2) {
        const float ur = re[off], ui = im[off], vr = re[off + 1], vi = im[off + 1];
        re[off] = ur + vr;
        im[off] = ui + vi;
        re[off + 1] = ur - vr;
        im[off + 1] = ui - vi;
    } else if constexpr (L >= 4) {
        constexpr int Q = L / 4;
#pragma unroll
        for (int n = 0; n < Q; ++n) {
            const int a = off + n, b = a + Q, c = b + Q, d = c + Q;
            const float t1r = re[a] - re[c], t1i = im[a] - im[c];
            const float t2r = re[b] - re[d], t2i = im[b] - im[d];
            re[a] += re[c];
            im[a] += im[c];
            re[b] += re[d];
            im[b] += im[d];
            // forward: z1 = t1 - j t2, z3 = t1 + j t2
            float z1r = ADJ ? t1r - t2i : t1r + t2i, z1i = ADJ ? t1i + t2r : t1i - t2r;
            float z3r = ADJ ? t1r + t2i : t1r - t2i, z3i = ADJ ? t1i - t2r : t1i + t2r;
            rot_any<ADJ>(z1r, z1i, n, L, w);
            rot_any<ADJ>(z3r, z3i, 3 * n, L, w);
            re[c] = z1r;
            im[c] = z1i;
            re[d] = z3r;
            im[d] = z3i;
        }
        dft_split_radix<L / 2, ADJ>(re, im, off, w);
        dft_split_radix<L / 4, ADJ>(re, im, off + L / 2, w);
        dft_split_radix<L / 4, ADJ>(re, im, off + 3 * L / 4, w);
    }
}

// In-register R-point DFT of re/im[off .. off+R-1] (natural input order),
// decimation in frequency (split radix); output bin d lands in register
// off + brevc(d, log2 R).  All indices are compile-time after unrolling.
template <int R, bool ADJ, int E>
__device__ __forceinline__ void dft_regs(float (&re)[E], float (&im)[E], const int off,
                                         const W64& w) {
    dft_split_radix<R, ADJ>(re, im, off, w);
}

// In-register R-point DFT in the order of Eq. (6): the input must sit in
// bit-reversed register order (S of Eq. (6), a compile-time renaming done by
// the caller); then for i = 1..log2 R the rotation D(i) (omega^(i,q) on the
// lower half of every block of 2^i points) and the butterfly W(i) (sum and
// difference of the halves).  Output bin d lands in register off + d.
template <int R, bool ADJ, int E>
__device__ __forceinline__ void dft_regs_dit(float (&re)[E], float (&im)[E], const int off,
                                             const W64& w) {
#pragma unroll
    for (int span = 1; span < R; span <<= 1) {
#pragma unroll
        for (int base = 0; base < R; base += 2 * span) {
#pragma unroll
            for (int q = 0; q < span; ++q) {
                const int a = off + base + q;
                const int b = a + span;
                float vr = re[b], vi = im[b];
                rot_const<ADJ>(vr, vi, q, 2 * span, w);       // D(i)
                const float ur = re[a], ui = im[a];
                re[a] = ur + vr;                              // W(i)
                im[a] = ui + vi;
                re[b] = ur - vr;
                im[b] = ui - vi;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Step engine.  A sub-DFT of size N = 2^LOGN is run by T = N / E cooperating
// threads (E = 2^LOGE elements each) in up to three steps of radix
// 2^LR0, 2^LR1, 2^LR2 (LR0 + LR1 + LR2 = LOGN, unused steps 0).
//
// Logical layout before step s: index L = D + P_s * n_rem, where D (< P_s)
// collects the output digits already produced and n_rem (< M_s = N / P_s) the
// input digits still to be summed.  Step s takes R_s-point DFTs over the top
// digit of n_rem: column c = D + P_s * nl (nl < Q_s = M_s / R_s) holds
// elements L = c + C_s * i (C_s = N / R_s, i < R_s).  Output digit d of
// column c is rotated by W_{M_s}^{nl * d} and moves to
// L' = D + P_s * d + P_s * R_s * nl.  After the last step L' is the natural
// output index k.  Thread t owns columns c = t + T * f, f < E / R_s.
//
// The caller supplies:
//   ld(L, re, im)        step-0 input element L
//   xw(L, re, im)        write exchange element L     (steps < last)
//   xr(L, re, im)        read exchange element L      (steps > 0)
//   tw(s, d, nl) float2  W_{M_s}^{nl * d} for step s  (steps < last)
//   st(k, re, im)        output element k
//   sync()               barrier over the T threads of this sub-DFT (and
//                        every other sub-DFT sharing its exchange buffer)
// ---------------------------------------------------------------------------
template <int LOGN_, int LOGE_, int LR0, int LR1, int LR2, bool DIT_ = false>
struct Steps {
    // DIT: the register DFTs of every step run in the order of Eq. (6)
    // (bit-reversed gather, rotation then butterfly); otherwise decimation in
    // frequency (butterfly then rotation, bit-reversed result).  Same values
    // up to rounding order.
    static constexpr bool DIT = DIT_;
    static constexpr int LOGN = LOGN_, N = 1 << LOGN;
    static constexpr int LOGE = LOGE_, E = 1 << LOGE;
    static constexpr int LOGT = LOGN - LOGE, T = 1 << LOGT;
    static constexpr int NS = (LR0 > 0) + (LR1 > 0) + (LR2 > 0);
    static_assert(LR0 + LR1 + LR2 == LOGN, "radices must multiply to N");
    static_assert(LR0 > 0 && (LR1 > 0 || LR2 == 0), "steps must be packed");
    static_assert(LR0 <= LOGE && LR1 <= LOGE && LR2 <= LOGE, "radix exceeds registers");
    static_assert(LOGE <= 6, "at most 64 elements per thread");
    __host__ __device__ static constexpr int lr(int s) { return s == 0 ? LR0 : s == 1 ? LR1 : LR2; }
    __host__ __device__ static constexpr int lp(int s) { return s == 0 ? 0 : s == 1 ? LR0 : LR0 + LR1; }
    // twiddle-table entries of step s (M_s = N / P_s)
    __host__ __device__ static constexpr int tw_entries(int s) { return N >> lp(s); }
};

template <class S, int s>
struct StepK {
    static constexpr int LR = S::lr(s), R = 1 << LR;
    static constexpr int LP = S::lp(s), P = 1 << LP;
    static constexpr int LM = S::LOGN - LP, M = 1 << LM;
    static constexpr int LQ = LM - LR, Q = 1 << LQ;
    static constexpr int F = S::E / R;
    static constexpr int LC = S::LOGN - LR, C = 1 << LC;
    static constexpr bool LAST = (s == S::NS - 1);
};

template <class S, int s, bool ADJ, class XR, class LD>
__device__ __forceinline__ void step_gather(float (&re)[S::E], float (&im)[S::E], const int t,
                                            LD& ld, XR& xr) {
    using K = StepK<S, s>;
#pragma unroll
    for (int f = 0; f < K::F; ++f)
#pragma unroll
        for (int i = 0; i < K::R; ++i) {
            const int L = t + S::T * f + K::C * i;
            const int reg = f * K::R + (S::DIT ? brevc(i, K::LR) : i);
            if constexpr (s == 0) ld(L, re[reg], im[reg]);
            else xr(L, re[reg], im[reg]);
        }
}

// The register DFTs of step s (no memory access).
template <class S, int s, bool ADJ>
__device__ __forceinline__ void step_compute(float (&re)[S::E], float (&im)[S::E], const W64& w) {
    using K = StepK<S, s>;
#pragma unroll
    for (int f = 0; f < K::F; ++f) {
        if constexpr (S::DIT) dft_regs_dit<K::R, ADJ>(re, im, f * K::R, w);
        else dft_regs<K::R, ADJ>(re, im, f * K::R, w);
    }
}

// The rotations and exchange writes (or, for the last step, output stores)
// of step s.
template <class S, int s, bool ADJ, class TW, class XW, class ST>
__device__ __forceinline__ void step_scatter(float (&re)[S::E], float (&im)[S::E], const int t,
                                             TW& tw, XW& xw, ST& st) {
    using K = StepK<S, s>;
#pragma unroll
    for (int f = 0; f < K::F; ++f) {
        const int c = t + S::T * f;
        const int lo = c & (K::P - 1);
        const int nl = c >> K::LP;
#pragma unroll
        for (int d = 0; d < K::R; ++d) {
            const int reg = f * K::R + (S::DIT ? d : brevc(d, K::LR));
            if constexpr (K::LAST) {
                st(lo + K::P * d, re[reg], im[reg]);
            } else {
                if (d != 0) rot<ADJ>(re[reg], im[reg], tw(s, d, nl));
                xw(lo + K::P * d + K::P * K::R * nl, re[reg], im[reg]);
            }
        }
    }
}

template <class S, int s, bool ADJ, class TW, class XW, class ST>
__device__ __forceinline__ void step_compute_scatter(float (&re)[S::E], float (&im)[S::E],
                                                     const int t, const W64& w, TW& tw, XW& xw,
                                                     ST& st) {
    step_compute<S, s, ADJ>(re, im, w);
    step_scatter<S, s, ADJ>(re, im, t, tw, xw, st);
}

// Run all steps of S.  `sync` separates exchange writes from reads (and the
// reads of one step from the writes of the next).  SYNC0: also synchronise
// between the step-0 gather and the step-0 scatter, for callers whose step-0
// source and exchange buffer share shared memory.
template <class S, bool ADJ, bool SYNC0 = false, class LD, class XW, class XR, class TW, class ST,
          class SYNC>
__device__ __forceinline__ void run_steps(const int t, const W64& w, LD ld, XW xw, XR xr, TW tw,
                                          ST st, SYNC sync) {
    float re[S::E], im[S::E];
    step_gather<S, 0, ADJ>(re, im, t, ld, xr);
    if constexpr (SYNC0) sync();
    step_compute_scatter<S, 0, ADJ>(re, im, t, w, tw, xw, st);
    if constexpr (S::NS > 1) {
        sync();
        step_gather<S, 1, ADJ>(re, im, t, ld, xr);
        if constexpr (S::NS > 2) {
            sync();  // all reads of step 1 done before step 1 overwrites
        }
        step_compute_scatter<S, 1, ADJ>(re, im, t, w, tw, xw, st);
        if constexpr (S::NS > 2) {
            sync();
            step_gather<S, 2, ADJ>(re, im, t, ld, xr);
            step_compute_scatter<S, 2, ADJ>(re, im, t, w, tw, xw, st);
        }
    }
}

// Shared-memory index of exchange element L: one pad word per 32 keeps
// stride-32 and stride-16 column writes free of bank conflicts.
__device__ __forceinline__ int pad32(int L) { return L + (L >> 5); }

// The same without padding: element L at L ^ ((L >> 5) & 31), i.e. each line
// of 32 words rotated by XOR with its line index.  A stride-32 column write
// (one element per lane, lanes 32 apart) then falls on 32 banks, as do reads
// of 32 consecutive elements; the exchange takes exactly N words per plane.
__device__ __forceinline__ int swz32(int L) { return L ^ ((L >> 5) & 31); }

}  // namespace sdft
