/*
 * tcbf_oracle.c — plain, slow, obviously correct CPU oracle for the
 * tensor-core beamformer (arXiv 2505.03269).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA path.
 *
 * Every routine is the definition written out with FP64 (or int64)
 * arithmetic and a sequential k loop per output element:
 *   - complex beamforming sum, Eq. 3 (Sec. II), M = beams, N = samples,
 *     K = receivers, with the complex product of Sec. III-B;
 *   - IEEE binary16 decoding (the library's FP16 storage format);
 *   - 1-bit complex values per Fig. 1 (bit 1 -> +1, bit 0 -> -1, one bit
 *     for the real and one for the imaginary part), unpacked and multiplied
 *     as explicit +-1 integers;
 *   - sign quantisation into those bits (Sec. III-D, Sec. V-A);
 *   - steering weights w = A exp(-2 pi i f tau) from geometry, Eq. 1-2.
 *
 * Layouts (all row-major, "interleaved" = (re, im) adjacent):
 *   W  [Bw][M][K] complex,  X [B][K][N] complex,  Y [B][M][N] complex.
 *   Batch b uses weight matrix b / (B / Bw).
 *   Packed 1-bit planes: [B][2][rows][Kw] uint32, plane 0 = real, plane 1 =
 *   imaginary, element k of a row is bit (k % 32) of word (k / 32).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the OpenMP loops below use (1 without OpenMP). */
EXPORT int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* IEEE 754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
EXPORT double oracle_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 31;
    int f = h & 1023;
    double v;
    if (e == 0)
        v = ldexp((double)f, -24);                   /* subnormal: f * 2^-24 */
    else if (e == 31)
        v = f ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + f), e - 25);       /* (1 + f/1024) * 2^(e-15) */
    return sign ? -v : v;
}

/* Eq. 3 on double inputs: Y[b,m,n] = sum_k W[b',m,k] * X[b,k,n]. */
EXPORT void oracle_cgemm_f64(int64_t B, int64_t M, int64_t N, int64_t K, int64_t Bw,
                             const double *W, const double *X, double *Y)
{
    const int64_t per_w = B / Bw;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        for (int64_t m = 0; m < M; ++m) {
            const double *w = W + ((b / per_w) * M + m) * K * 2;
            double *y = Y + (b * M + m) * N * 2;
            for (int64_t n = 0; n < N; ++n) {
                y[2 * n] = 0.0;
                y[2 * n + 1] = 0.0;
            }
            for (int64_t k = 0; k < K; ++k) {
                const double wr = w[2 * k], wi = w[2 * k + 1];
                const double *x = X + (b * K + k) * N * 2;
                for (int64_t n = 0; n < N; ++n) {
                    const double xr = x[2 * n], xi = x[2 * n + 1];
                    /* Re(ab) = Re a Re b - Im a Im b ; Im(ab) = Re a Im b + Im a Re b */
                    y[2 * n] += wr * xr - wi * xi;
                    y[2 * n + 1] += wr * xi + wi * xr;
                }
            }
        }
}

/* Eq. 3 on the library's FP16 inputs: each half is widened exactly to double
 * (per batch, once), then the same FP64 loops as above. Work buffers are
 * supplied by the caller: xd holds K*N*2 doubles per thread-free batch pass. */
EXPORT void oracle_cgemm_f16(int64_t B, int64_t M, int64_t N, int64_t K, int64_t Bw,
                             const uint16_t *W, const uint16_t *X, double *Y,
                             double *wd /* M*K*2 */, double *xd /* K*N*2 */)
{
    const int64_t per_w = B / Bw;
    int64_t w_loaded = -1;
    for (int64_t b = 0; b < B; ++b) {
        const int64_t bw = b / per_w;
        if (bw != w_loaded) {
            for (int64_t i = 0; i < M * K * 2; ++i)
                wd[i] = oracle_half_to_double(W[bw * M * K * 2 + i]);
            w_loaded = bw;
        }
        for (int64_t i = 0; i < K * N * 2; ++i)
            xd[i] = oracle_half_to_double(X[b * K * N * 2 + i]);
        oracle_cgemm_f64(1, M, N, K, 1, wd, xd, Y + b * M * N * 2);
    }
}

/* Eq. 3 at selected output points (b, m, n), FP16 inputs, one by one. */
EXPORT void oracle_cgemm_f16_points(int64_t B, int64_t M, int64_t N, int64_t K, int64_t Bw,
                                    const uint16_t *W, const uint16_t *X,
                                    int64_t npts, const int64_t *pts, double *out)
{
    const int64_t per_w = B / Bw;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npts; ++p) {
        const int64_t b = pts[3 * p], m = pts[3 * p + 1], n = pts[3 * p + 2];
        const uint16_t *w = W + ((b / per_w) * M + m) * K * 2;
        double re = 0.0, im = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            const uint16_t *x = X + ((b * K + k) * N + n) * 2;
            const double wr = oracle_half_to_double(w[2 * k]);
            const double wi = oracle_half_to_double(w[2 * k + 1]);
            const double xr = oracle_half_to_double(x[0]);
            const double xi = oracle_half_to_double(x[1]);
            re += wr * xr - wi * xi;
            im += wr * xi + wi * xr;
        }
        out[2 * p] = re;
        out[2 * p + 1] = im;
    }
}

/* Fig. 1: bit value 1 -> +1, 0 -> -1. Element k of a row sits in bit k%32 of word k/32. */
static int64_t onebit_value(const uint32_t *row, int64_t k)
{
    return ((row[k >> 5] >> (k & 31)) & 1u) ? 1 : -1;
}

/* Eq. 3 over 1-bit complex values (Sec. III-D), exact in int64.
 * Wb [Bw][2][M][Kw], Xb [B][2][N][Kw] (X stored with samples as rows),
 * Y [B][M][N][2] int64. Bits at k >= K are ignored. */
EXPORT void oracle_bgemm(int64_t B, int64_t M, int64_t N, int64_t K, int64_t Bw, int64_t Kw,
                         const uint32_t *Wb, const uint32_t *Xb, int64_t *Y)
{
    const int64_t per_w = B / Bw;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int64_t b = 0; b < B; ++b)
        for (int64_t m = 0; m < M; ++m) {
            const int64_t bw = b / per_w;
            const uint32_t *wr_row = Wb + ((bw * 2 + 0) * M + m) * Kw;
            const uint32_t *wi_row = Wb + ((bw * 2 + 1) * M + m) * Kw;
            for (int64_t n = 0; n < N; ++n) {
                const uint32_t *xr_row = Xb + ((b * 2 + 0) * N + n) * Kw;
                const uint32_t *xi_row = Xb + ((b * 2 + 1) * N + n) * Kw;
                int64_t re = 0, im = 0;
                for (int64_t k = 0; k < K; ++k) {
                    const int64_t ar = onebit_value(wr_row, k), ai = onebit_value(wi_row, k);
                    const int64_t br = onebit_value(xr_row, k), bi = onebit_value(xi_row, k);
                    re += ar * br - ai * bi;
                    im += ar * bi + ai * br;
                }
                Y[((b * M + m) * N + n) * 2] = re;
                Y[((b * M + m) * N + n) * 2 + 1] = im;
            }
        }
}

/* 1-bit sample of one real value (Sec. III-D: zero is not representable):
 * the bit keeps the sign, 1 for v >= 0 (so +0 and -0 give +1), 0 otherwise. */
static uint32_t sign_bit(double v)
{
    return v >= 0.0 ? 1u : 0u;
}

/* Sign-quantise interleaved complex FP16 rows into packed planes.
 * src is [B][R][C] complex.  When k_is_row is 0 the packed axis (the GEMM's
 * K) is C, so out[b][p][r][w] packs src[b][r][k]; when it is 1 the packed
 * axis is R and out[b][p][c][w] packs src[b][k][c] (a transpose).
 * Words are Kw long; bits for k >= K are 0. */
EXPORT void oracle_pack_signs_f16(int64_t B, int64_t R, int64_t C, int k_is_row, int64_t Kw,
                                  const uint16_t *src, uint32_t *out)
{
    const int64_t K = k_is_row ? R : C;
    const int64_t rows = k_is_row ? C : R;
    memset(out, 0, (size_t)(B * 2 * rows * Kw) * sizeof(uint32_t));
    for (int64_t b = 0; b < B; ++b)
        for (int64_t r = 0; r < rows; ++r)
            for (int64_t k = 0; k < K; ++k) {
                const int64_t e = k_is_row ? ((b * R + k) * C + r) : ((b * R + r) * C + k);
                for (int p = 0; p < 2; ++p) {
                    const double v = oracle_half_to_double(src[2 * e + p]);
                    out[((b * 2 + p) * rows + r) * Kw + (k >> 5)] |= sign_bit(v) << (k & 31);
                }
            }
}

/* Steering weights, Eq. 1-2 with the delay compensated by the weight:
 *   far field : tau = (p_k . s_m) / c,  A = 1          (s_m a unit direction)
 *   near field: d = |t_m - p_k|, tau = d / c, A = 1 / d (t_m a target position)
 *   w[b,m,k] = A * exp(-2 pi i f[b,k] tau) = A cos(2 pi f tau) - i A sin(2 pi f tau).
 * rx [K][3], tg [M][3], freqs [Bw][K], out [Bw][M][K] interleaved doubles. */
EXPORT void oracle_weights(int64_t Bw, int64_t M, int64_t K, const double *rx, const double *tg,
                           int near_field, const double *freqs, double c, double *out)
{
    const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t b = 0; b < Bw; ++b)
        for (int64_t m = 0; m < M; ++m)
            for (int64_t k = 0; k < K; ++k) {
                double tau, amp;
                if (near_field) {
                    const double dx = tg[3 * m] - rx[3 * k];
                    const double dy = tg[3 * m + 1] - rx[3 * k + 1];
                    const double dz = tg[3 * m + 2] - rx[3 * k + 2];
                    const double d = sqrt(dx * dx + dy * dy + dz * dz);
                    tau = d / c;
                    amp = 1.0 / d;
                } else {
                    tau = (rx[3 * k] * tg[3 * m] + rx[3 * k + 1] * tg[3 * m + 1] +
                           rx[3 * k + 2] * tg[3 * m + 2]) / c;
                    amp = 1.0;
                }
                const double phase = two_pi * (freqs[b * K + k] * tau);
                out[((b * M + m) * K + k) * 2] = amp * cos(phase);
                out[((b * M + m) * K + k) * 2 + 1] = -amp * sin(phase);
            }
}

/* ------------------------------------------------------------------------
 * Split-FP8 (the paper names 8-bit float formats as future work, Sec. VI).
 * E4M3: 1 sign bit, 4 exponent bits (bias 7), 3 fraction bits; normal values
 * (1 + f/8) 2^(E-7) for E = 1..15 (largest finite 448 = 1.75 * 2^8, the code
 * with E = 15 and f = 7 being NaN), subnormals (f/8) 2^-6.  Rounding is to
 * the nearest representable value, ties to an even fraction; magnitudes
 * beyond 448 saturate to 448.
 * ---------------------------------------------------------------------- */
EXPORT double oracle_e4m3_round(double v)
{
    if (v != v) return v;
    const double a = fabs(v);
    if (a >= 448.0) return v < 0 ? -448.0 : 448.0;
    if (a == 0.0) return v;
    int q;
    frexp(a, &q);                      /* a = m 2^q, m in [0.5, 1): a in [2^(q-1), 2^q) */
    int e = q - 1;                     /* a in [2^e, 2^(e+1)) */
    if (e < -6) e = -6;                /* subnormal range shares the spacing of 2^-6 */
    const double ulp = ldexp(1.0, e - 3);
    const double n = a / ulp;          /* exact: a power-of-two scaling */
    double r = floor(n);
    const double frac = n - r;
    if (frac > 0.5 || (frac == 0.5 && fmod(r, 2.0) != 0.0)) r += 1.0;
    double out = r * ulp;
    if (out > 448.0) out = 448.0;
    return v < 0 ? -out : out;
}

/* The largest integer e with amax * 2^e <= 448 (0 for amax == 0). */
EXPORT int oracle_split_exponent(double amax)
{
    if (!(amax > 0.0)) return 0;
    int e = (int)floor(log2(448.0 / amax));
    while (ldexp(amax, e) > 448.0) --e;
    while (ldexp(amax, e + 1) <= 448.0) ++e;
    return e;
}

/* Split rows of interleaved complex FP16 values into E4M3 hi and lo parts:
 * per row (over k < K and both planes) the scale exponent e, then
 * hi = RN(v 2^e), lo = RN(v 2^e - hi).  rows: [R][K] complex;
 * hi, lo: [R][K][2] doubles (scaled values); exps: [R]. */
EXPORT void oracle_split_rows(int64_t R, int64_t K, const uint16_t *src, double *hi, double *lo,
                              int32_t *exps)
{
    for (int64_t r = 0; r < R; ++r) {
        double amax = 0.0;
        for (int64_t i = 0; i < 2 * K; ++i) {
            const double a = fabs(oracle_half_to_double(src[r * 2 * K + i]));
            if (a > amax) amax = a;
        }
        const int e = oracle_split_exponent(amax);
        exps[r] = e;
        for (int64_t i = 0; i < 2 * K; ++i) {
            const double v = ldexp(oracle_half_to_double(src[r * 2 * K + i]), e);
            const double h = oracle_e4m3_round(v);
            hi[r * 2 * K + i] = h;
            lo[r * 2 * K + i] = oracle_e4m3_round(v - h);
        }
    }
}

/* Block-scaled split (the FP8 forms' per-tile scales): per row and per block
 * of 32 consecutive k (over both planes) the exponent e of the block's
 * largest magnitude as above, hi = RN(v 2^e) and lo = RN(16 (v 2^e - hi)):
 * the lo part is stored 16 times larger (its scale is 2^-(e + 4)) so that it
 * keeps E4M3's precision.  rows: [R][K] complex; hi, lo: [R][K][2] doubles
 * (scaled values); exps: [R][ceil(K / 32)]. */
EXPORT void oracle_split_blocks(int64_t R, int64_t K, const uint16_t *src, double *hi, double *lo,
                                int32_t *exps)
{
    const int64_t nblk = (K + 31) / 32;
    for (int64_t r = 0; r < R; ++r)
        for (int64_t j = 0; j < nblk; ++j) {
            const int64_t k0 = 32 * j, k1 = k0 + 32 < K ? k0 + 32 : K;
            double amax = 0.0;
            for (int64_t i = 2 * k0; i < 2 * k1; ++i) {
                const double a = fabs(oracle_half_to_double(src[r * 2 * K + i]));
                if (a > amax) amax = a;
            }
            const int e = oracle_split_exponent(amax);
            exps[r * nblk + j] = e;
            for (int64_t i = 2 * k0; i < 2 * k1; ++i) {
                const double v = ldexp(oracle_half_to_double(src[r * 2 * K + i]), e);
                const double h = oracle_e4m3_round(v);
                hi[r * 2 * K + i] = h;
                lo[r * 2 * K + i] = oracle_e4m3_round(16.0 * (v - h));
            }
        }
}

