/*
 * sdft_oracle.c -- CPU oracle for the split (planar) complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may build, load or call
 * it.  The CUDA library never links it, and it includes nothing from the CUDA
 * library (no shared headers, tables or helpers).
 *
 * Paper: A. Cariow, "Fast algorithms for complex-valued discrete Fourier
 * transform with separate real and imaginary inputs/outputs" (arXiv 2504.07264).
 *
 * Everything is IEEE binary64, compiled without fast-math and without FMA
 * contraction, so x86-64 and aarch64 hosts produce the same numbers.
 *
 * Arrays are planar and row-major: row b of a batch is xr[b*n .. b*n+n-1]
 * (real parts) and xi[b*n .. ] (imaginary parts); outputs likewise.
 *
 * Functions:
 *   O1  sdft_oracle_direct          Eq. (1), written in the split form Eq. (3):
 *                                   y^r = C x^r + S x^i,  y^i = C x^i - S x^r.
 *   O1b sdft_oracle_direct_bins     the same, evaluated on a chosen set of bins.
 *   O2  sdft_oracle_factored_dit    the vector-matrix procedure Eq. (6):
 *                                   y = W(m) D(m) ... W(1) D(1) S x  (Section III).
 *   O2s sdft_oracle_dit_stages      Eq. (6) on one transform, recording the
 *                                   vector after S and after every D(i), W(i).
 *   O3  sdft_oracle_adjoint_direct  the transposed block matrix of Eq. (5):
 *                                   E^T = [C -S; S C] on [x^r; x^i].
 *   O3f sdft_oracle_adjoint_factored the transpose of the Eq. (6) product,
 *                                   S^T D(1)^T W(1)^T ... D(m)^T W(m)^T x.
 *   O4  sdft_oracle_factored_dif    the decimation-in-frequency procedure Eq. (9):
 *                                   y = S D(1) W(1) ... D(m) W(m) x.
 *   O2f sdft_oracle_factored_dit_f32 Eq. (6) carried out in binary32 (the CPU
 *                                   baseline's single-precision instance; each
 *                                   omega^(i,q) entry rounded once from
 *                                   binary64).  Checked against O2, not a
 *                                   parity oracle itself.
 *
 * Readings of the paper taken here:
 *   - Eq. (2) prints y = E y; the intended map is y = E x.
 *   - In the definitions under Eq. (6) the leading identity of W(i) and D(i)
 *     is printed as I_{2^{m-1}}; its order must be 2^{m-i} for the Kronecker
 *     product to have order 2^{m+1}, and the N = 8 example (Eq. (7)) uses
 *     2^{3-i}.  The code uses I_{2^{m-i}}.
 *   - The example's omega^(3,3) (Eq. (8)) is printed equal to omega^(3,1);
 *     the defining formula under Eq. (6) is used for every omega^(i,q).
 *   - N = 2^m; Section III states m >= 2, the formulas also hold for m = 1
 *     and m = 0 is the identity map, both accepted here.
 *   - No normalisation anywhere (Eq. (1) has none).
 *
 * Every entry point takes `threads`: the number of OpenMP threads over the
 * independent transforms of a batch (0 = the OpenMP default).  Threading
 * never changes the arithmetic of a single transform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double TWO_PI = 6.283185307179586476925286766559;

/* ---- mutation hooks: compiled in only when a test asks for a planted
 * mistake (-DSDFT_ORACLE_MUTATION=k); the default build has none. ---- */
#ifndef SDFT_ORACLE_MUTATION
#define SDFT_ORACLE_MUTATION 0
#endif

static int set_threads(int threads) {
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* log2 of a power of two; -1 if n is not one. */
static int ilog2_exact(int64_t n) {
    if (n < 1) return -1;
    int m = 0;
    while (((int64_t)1 << m) < n) ++m;
    return (((int64_t)1 << m) == n) ? m : -1;
}

/* <n>_2: reverse the m low bits of n (Section III, definition of S_{2^m}). */
static int64_t bit_reverse(int64_t n, int m) {
    int64_t r = 0;
    for (int i = 0; i < m; ++i) {
        int64_t bit = (n >> i) & 1;          /* n_i */
        r |= bit << (m - 1 - i);             /* placed at position m-1-i */
    }
    return r;
}

/* cos and sin of 2 pi r / n.  At quarter turns (4r divisible by n) the
 * entries c_{k,n}, s_{k,n} of Eq. (3) and the omega^(i,q) blocks are exactly
 * 0 and +-1; they are returned exactly there (libm's sin(pi) is 1.2e-16, not
 * 0) and taken from libm cos/sin everywhere else. */
static void cos_sin_turn(int64_t r, int64_t n, double* c, double* s) {
    r %= n;
    if ((4 * r) % n == 0) {
        static const double C[4] = {1.0, 0.0, -1.0, 0.0};
        static const double S[4] = {0.0, 1.0, 0.0, -1.0};
        int q = (int)((4 * r) / n) & 3;
        *c = C[q];
        *s = S[q];
        return;
    }
    double ang = TWO_PI * (double)r / (double)n;
    *c = cos(ang);
    *s = sin(ang);
}

/* ------------------------------------------------------------------ O1 -- */
/* One bin of Eq. (3): y_k^r = sum_n (x_n^r c_{k,n} + x_n^i s_{k,n}),
 *                     y_k^i = sum_n (x_n^i c_{k,n} - x_n^r s_{k,n}),
 * with c_{k,n} = cos(2 pi k n / N), s_{k,n} = sin(2 pi k n / N).  The product
 * k*n is reduced modulo N in integers first, so the angle is exact before the
 * library cos/sin is applied. */
static void direct_bin(int64_t n, int64_t k, const double* xr, const double* xi,
                       double* out_r, double* out_i) {
    double acc_r = 0.0, acc_i = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t r = (k * t) % n;
        double c, s;
        cos_sin_turn(r, n, &c, &s);
#if SDFT_ORACLE_MUTATION == 1
        s = -s;                               /* planted: wrong sign of S */
#endif
        acc_r += xr[t] * c + xi[t] * s;
        acc_i += xi[t] * c - xr[t] * s;
    }
    *out_r = acc_r;
    *out_i = acc_i;
}

int sdft_oracle_direct(int64_t n, int64_t batch, const double* xr, const double* xi,
                       double* yr, double* yi, int threads) {
    if (n < 1 || batch < 0) return -1;
    int nt = set_threads(threads);
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t b = 0; b < batch; ++b) {
        const double* ar = xr + b * n;
        const double* ai = xi + b * n;
        for (int64_t k = 0; k < n; ++k)
            direct_bin(n, k, ar, ai, yr + b * n + k, yi + b * n + k);
    }
    return 0;
}

/* Eq. (3) on nbins chosen bins per transform: out[b*nbins + j] = y_{bins[j]}. */
int sdft_oracle_direct_bins(int64_t n, int64_t batch, const double* xr, const double* xi,
                            const int64_t* bins, int64_t nbins,
                            double* yr, double* yi, int threads) {
    if (n < 1 || batch < 0 || nbins < 0) return -1;
    for (int64_t j = 0; j < nbins; ++j)
        if (bins[j] < 0 || bins[j] >= n) return -1;
    int nt = set_threads(threads);
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t b = 0; b < batch; ++b)
        for (int64_t j = 0; j < nbins; ++j)
            direct_bin(n, bins[j], xr + b * n, xi + b * n,
                       yr + b * nbins + j, yi + b * nbins + j);
    return 0;
}

/* ------------------------------------------------- factors of Eq. (6) -- */
/* The procedure works on the interleaved pair vector of Section III,
 * x_2N = [x0^r, x0^i, x1^r, x1^i, ...], of length 2^{m+1}. */

/* S_{2^{m+1}} = S_{2^m} (x) I_2: entry pair k of the result is pair <k>_2 of
 * the input (each row k of S_{2^m} has its one in column <k>_2). */
static void apply_S(int m, const double* in, double* out) {
    int64_t N = (int64_t)1 << m;
    for (int64_t k = 0; k < N; ++k) {
        int64_t src = bit_reverse(k, m);
#if SDFT_ORACLE_MUTATION == 3
        src = k;                              /* planted: permutation dropped */
#endif
        out[2 * k] = in[2 * src];
        out[2 * k + 1] = in[2 * src + 1];
    }
}

/* W(i) = I_{2^{m-i}} (x) H_2 (x) I_{2^i}, H_2 = [1 1; 1 -1]: in every block of
 * 2^{i+1} entries, entry j and entry j + 2^i (j < 2^i) become (u+v, u-v). */
static void apply_W(int m, int i, double* v) {
    int64_t len = (int64_t)2 << m;            /* 2^{m+1} */
    int64_t half = (int64_t)1 << i;           /* 2^i */
    for (int64_t base = 0; base < len; base += 2 * half)
        for (int64_t j = 0; j < half; ++j) {
            double u = v[base + j], w = v[base + j + half];
            v[base + j] = u + w;
            v[base + j + half] = u - w;
        }
}

/* omega^(i,q) = [cos t  sin t; -sin t  cos t], t = 2 pi q / 2^i, applied to the
 * column (a, b); transpose != 0 applies its transpose [cos -sin; sin cos]. */
static void apply_omega(int i, int64_t q, double* pair, int transpose) {
    double c, s;
    cos_sin_turn(q, (int64_t)1 << i, &c, &s);
#if SDFT_ORACLE_MUTATION == 2
    s = -s;                                   /* planted: conjugated twiddle */
#endif
    double a = pair[0], b = pair[1];
    if (!transpose) {
        pair[0] = c * a + s * b;
        pair[1] = -s * a + c * b;
    } else {
        pair[0] = c * a - s * b;
        pair[1] = s * a + c * b;
    }
}

/* D(i) = I_{2^{m-i}} (x) D_{2^{i+1}},
 * D_{2^{i+1}} = diag(I_{2R}, omega^(i,0), ..., omega^(i,R-1)), R = 2^{i-1}:
 * in every block of 2^{i+1} entries the first 2R entries pass unchanged and
 * pair q of the last 2R entries is multiplied by omega^(i,q). */
static void apply_D(int m, int i, double* v, int transpose) {
    int64_t len = (int64_t)2 << m;
    int64_t block = (int64_t)2 << i;          /* 2^{i+1} entries */
    int64_t R = (int64_t)1 << (i - 1);
    for (int64_t base = 0; base < len; base += block)
        for (int64_t q = 0; q < R; ++q) {
#if SDFT_ORACLE_MUTATION == 4
            apply_omega(i, q, v + base + 2 * q, transpose);   /* planted: top half */
#else
            apply_omega(i, q, v + base + 2 * R + 2 * q, transpose);
#endif
        }
}

static void planar_to_pairs(int64_t n, const double* xr, const double* xi, double* v) {
    for (int64_t k = 0; k < n; ++k) {
        v[2 * k] = xr[k];
        v[2 * k + 1] = xi[k];
    }
}

static void pairs_to_planar(int64_t n, const double* v, double* yr, double* yi) {
    for (int64_t k = 0; k < n; ++k) {
        yr[k] = v[2 * k];
        yi[k] = v[2 * k + 1];
    }
}

/* ------------------------------------------------------------------ O2 -- */
/* Eq. (6): y = W(m) D(m) ... W(1) D(1) S x, applied right to left. */
static void dit_one(int m, const double* xr, const double* xi, double* yr, double* yi,
                    double* v, double* tmp) {
    int64_t N = (int64_t)1 << m;
    planar_to_pairs(N, xr, xi, tmp);
    apply_S(m, tmp, v);
    for (int i = 1; i <= m; ++i) {
        apply_D(m, i, v, 0);
        apply_W(m, i, v);
    }
    pairs_to_planar(N, v, yr, yi);
}

int sdft_oracle_factored_dit(int64_t n, int64_t batch, const double* xr, const double* xi,
                             double* yr, double* yi, int threads) {
    int m = ilog2_exact(n);
    if (m < 0 || batch < 0) return -1;
    int nt = set_threads(threads);
    int fail = 0;
    #pragma omp parallel num_threads(nt) reduction(|: fail)
    {
        double* v = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        if (!v || !tmp) {
            fail = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t b = 0; b < batch; ++b)
                dit_one(m, xr + b * n, xi + b * n, yr + b * n, yi + b * n, v, tmp);
        }
        free(v);
        free(tmp);
    }
    return fail ? -2 : 0;
}

/* ----------------------------------------------------------------- O2f -- */
/* Eq. (6) in binary32: S, then D(i) and W(i) for i = 1..m on a float pair
 * vector, the same index sets as apply_S / apply_D / apply_W.  Each
 * omega^(i,q) entry is cos/sin of the exact turn q / 2^i in binary64,
 * rounded once to binary32; every product and sum is a binary32 operation. */
static void dit_one_f32(int m, const float* xr, const float* xi, float* yr, float* yi,
                        float* v) {
    int64_t N = (int64_t)1 << m, len = (int64_t)2 << m;
    for (int64_t k = 0; k < N; ++k) {                      /* S */
        int64_t src = bit_reverse(k, m);
        v[2 * k] = xr[src];
        v[2 * k + 1] = xi[src];
    }
    for (int i = 1; i <= m; ++i) {
        int64_t block = (int64_t)2 << i, R = (int64_t)1 << (i - 1), half = (int64_t)1 << i;
        for (int64_t base = 0; base < len; base += block)  /* D(i): lower half of each block */
            for (int64_t q = 0; q < R; ++q) {
                double c, s;
                cos_sin_turn(q, (int64_t)1 << i, &c, &s);
                float cf = (float)c, sf = (float)s;
                float* pr = v + base + 2 * R + 2 * q;
                float a = pr[0], b = pr[1];
                pr[0] = cf * a + sf * b;
                pr[1] = -sf * a + cf * b;
            }
        for (int64_t base = 0; base < len; base += 2 * half)   /* W(i) */
            for (int64_t j = 0; j < half; ++j) {
                float u = v[base + j], w = v[base + j + half];
                v[base + j] = u + w;
                v[base + j + half] = u - w;
            }
    }
    for (int64_t k = 0; k < N; ++k) {
        yr[k] = v[2 * k];
        yi[k] = v[2 * k + 1];
    }
}

int sdft_oracle_factored_dit_f32(int64_t n, int64_t batch, const float* xr, const float* xi,
                                 float* yr, float* yi, int threads) {
    int m = ilog2_exact(n);
    if (m < 0 || batch < 0) return -1;
    int nt = set_threads(threads);
    int fail = 0;
    #pragma omp parallel num_threads(nt) reduction(|: fail)
    {
        float* v = (float*)malloc(sizeof(float) * 2 * (size_t)n);
        if (!v) {
            fail = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t b = 0; b < batch; ++b)
                dit_one_f32(m, xr + b * n, xi + b * n, yr + b * n, yi + b * n, v);
        }
        free(v);
    }
    return fail ? -2 : 0;
}

/* Eq. (6) on one transform, recording every intermediate pair vector:
 * stages[0] = S x, then for i = 1..m: stages[2i-1] = D(i) (...),
 * stages[2i] = W(i) (...).  `stages` holds (2m+1) vectors of 2N doubles;
 * `x2` is the interleaved input of Section III. */
int sdft_oracle_dit_stages(int64_t n, const double* x2, double* stages) {
    int m = ilog2_exact(n);
    if (m < 0) return -1;
    int64_t len = 2 * n;
    apply_S(m, x2, stages);
    for (int i = 1; i <= m; ++i) {
        double* d = stages + (2 * i - 1) * len;
        memcpy(d, d - len, sizeof(double) * (size_t)len);
        apply_D(m, i, d, 0);
        double* w = stages + (2 * i) * len;
        memcpy(w, d, sizeof(double) * (size_t)len);
        apply_W(m, i, w);
    }
    return 0;
}

/* ------------------------------------------------------------------ O4 -- */
/* Eq. (9): y = S D(1) W(1) ... D(m) W(m) x, applied right to left: W(m) first,
 * S last.  The same (untransposed) D(i) as Eq. (6). */
static void dif_one(int m, const double* xr, const double* xi, double* yr, double* yi,
                    double* v, double* tmp) {
    int64_t N = (int64_t)1 << m;
    planar_to_pairs(N, xr, xi, v);
    for (int i = m; i >= 1; --i) {
        apply_W(m, i, v);
        apply_D(m, i, v, 0);
    }
    apply_S(m, v, tmp);
    pairs_to_planar(N, tmp, yr, yi);
}

int sdft_oracle_factored_dif(int64_t n, int64_t batch, const double* xr, const double* xi,
                             double* yr, double* yi, int threads) {
    int m = ilog2_exact(n);
    if (m < 0 || batch < 0) return -1;
    int nt = set_threads(threads);
    int fail = 0;
    #pragma omp parallel num_threads(nt) reduction(|: fail)
    {
        double* v = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        if (!v || !tmp) {
            fail = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t b = 0; b < batch; ++b)
                dif_one(m, xr + b * n, xi + b * n, yr + b * n, yi + b * n, v, tmp);
        }
        free(v);
        free(tmp);
    }
    return fail ? -2 : 0;
}

/* ------------------------------------------------------------------ O3 -- */
/* E_2N^T applied to [x^r; x^i] with E_2N = [C S; -S C] (Eqs. (4)-(5)):
 * y^r = C x^r - S x^i,  y^i = S x^r + C x^i  (C and S are symmetric). */
int sdft_oracle_adjoint_direct(int64_t n, int64_t batch, const double* xr, const double* xi,
                               double* yr, double* yi, int threads) {
    if (n < 1 || batch < 0) return -1;
    int nt = set_threads(threads);
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t b = 0; b < batch; ++b) {
        const double* ar = xr + b * n;
        const double* ai = xi + b * n;
        for (int64_t k = 0; k < n; ++k) {
            double acc_r = 0.0, acc_i = 0.0;
            for (int64_t t = 0; t < n; ++t) {
                int64_t r = (k * t) % n;
                double c, s;
                cos_sin_turn(r, n, &c, &s);
#if SDFT_ORACLE_MUTATION == 5
                s = -s;                       /* planted: forward, not transpose */
#endif
                acc_r += c * ar[t] - s * ai[t];
                acc_i += s * ar[t] + c * ai[t];
            }
            yr[b * n + k] = acc_r;
            yi[b * n + k] = acc_i;
        }
    }
    return 0;
}

/* Transpose of the Eq. (6) product: (W(m) D(m) ... W(1) D(1) S)^T
 *   = S^T D(1)^T W(1)^T ... D(m)^T W(m)^T.
 * W(i) and S are symmetric, so applied right to left this is: W(m), D(m)^T,
 * ..., W(1), D(1)^T, then S. */
static void adjoint_factored_one(int m, const double* xr, const double* xi,
                                 double* yr, double* yi, double* v, double* tmp) {
    int64_t N = (int64_t)1 << m;
    planar_to_pairs(N, xr, xi, v);
    for (int i = m; i >= 1; --i) {
        apply_W(m, i, v);
        apply_D(m, i, v, 1);
    }
    apply_S(m, v, tmp);
    pairs_to_planar(N, tmp, yr, yi);
}

int sdft_oracle_adjoint_factored(int64_t n, int64_t batch, const double* xr, const double* xi,
                                 double* yr, double* yi, int threads) {
    int m = ilog2_exact(n);
    if (m < 0 || batch < 0) return -1;
    int nt = set_threads(threads);
    int fail = 0;
    #pragma omp parallel num_threads(nt) reduction(|: fail)
    {
        double* v = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)n);
        if (!v || !tmp) {
            fail = 1;
        } else {
            #pragma omp for schedule(dynamic, 1)
            for (int64_t b = 0; b < batch; ++b)
                adjoint_factored_one(m, xr + b * n, xi + b * n, yr + b * n, yi + b * n, v, tmp);
        }
        free(v);
        free(tmp);
    }
    return fail ? -2 : 0;
}

/* Number of OpenMP threads a call with `threads` uses (for reporting). */
int sdft_oracle_thread_count(int threads) { return set_threads(threads); }
