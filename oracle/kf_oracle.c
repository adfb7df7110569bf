/*
 * FP64 CPU oracle for fused BLAS-1/BLAS-2 sequences.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Every routine is the plain definition of what a sequence computes
 * (Filipovic et al., "Optimizing CUDA Code By Kernel Fusion -- Application
 * on BLAS", Table 1 of Section 4.1), evaluated in double precision on the
 * exact FP32 input values, with the script's sequential semantics (Section
 * 3.1: the script defines the order of calls and their data dependencies).
 *
 * Conventions:
 *   - A is m x n, row major, leading dimension lda >= n (elements);
 *   - A_ij is A[i * lda + j];
 *   - "Ap" is a length-m vector, "A^T r" a length-n vector.  (The paper's
 *     Section 3.4 text gives p, s the length m; its listing and Algorithm 3
 *     index p, s by column tiles and q, r by row tiles, which is the reading
 *     used here: p, s in R^n and q, r in R^m.)
 *
 * Inputs are double arrays holding FP32 values (the conversion is exact);
 * outputs are double arrays.  Intermediates stay in double.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* ---------------- BLAS-2 elementaries (Section 3.3, Eqs. 1-2) ---------- */

/* y_i = alpha * sum_j A_ij x_j + beta * y0_i   (y0 may be NULL if beta == 0)
 * The nested map(reduce(+, map(*, A_i, x)), A) form of GEMV, Section 3.3. */
void kfo_gemv(int64_t m, int64_t n, const double* A, int64_t lda,
              const double* x, double alpha, double beta, const double* y0,
              double* y) {
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) acc += A[i * lda + j] * x[j];
        y[i] = alpha * acc + (beta != 0.0 ? beta * y0[i] : 0.0);
    }
}

/* x_j = alpha * sum_i A_ij y_i + beta * x0_j : GEMV on A viewed as a list of
 * columns (Section 3.3, last paragraph). */
void kfo_gemvt(int64_t m, int64_t n, const double* A, int64_t lda,
               const double* y, double alpha, double beta, const double* x0,
               double* x) {
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t i = 0; i < m; ++i) acc += A[i * lda + j] * y[i];
        x[j] = alpha * acc + (beta != 0.0 ? beta * x0[j] : 0.0);
    }
}

/* B_ij = A_ij + alpha * u_i v_j (rank-1 update; B may equal A). */
void kfo_ger(int64_t m, int64_t n, const double* A, int64_t lda, double alpha,
             const double* u, const double* v, double* B, int64_t ldb) {
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j)
            B[i * ldb + j] = A[i * lda + j] + alpha * u[i] * v[j];
}

/* C_ij = A_ij + B_ij (MADD, Table 1). */
void kfo_madd(int64_t m, int64_t n, const double* A, const double* B, double* C) {
    for (int64_t i = 0; i < m * n; ++i) C[i] = A[i] + B[i];
}

/* ---------------- BLAS-1 elementaries ---------------------------------- */

/* out = alpha * x + beta * y   (AXPY, SCAL, WAXPBY are special cases). */
void kfo_axpby(int64_t n, double alpha, const double* x, double beta,
               const double* y, double* out) {
    for (int64_t i = 0; i < n; ++i)
        out[i] = alpha * x[i] + (beta != 0.0 ? beta * y[i] : 0.0);
}

/* out = w + y + z (VADD, Table 1). */
void kfo_vadd3(int64_t n, const double* w, const double* y, const double* z,
               double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = w[i] + y[i] + z[i];
}

/* sum_i x_i y_i : map(*) followed by reduce(+) (Section 3.3, DOT). */
double kfo_dot(int64_t n, const double* x, const double* y) {
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += x[i] * y[i];
    return acc;
}

/* ---------------- The sequences of Table 1 ------------------------------ */

/* BiCGK (Section 3.4, Listing 1 and Algorithm 3; Table 1):
 *   q = A p  (q in R^m),   s = A^T r  (s in R^n). */
void kfo_bicgk(int64_t m, int64_t n, const double* A, int64_t lda,
               const double* p, const double* r, double* q, double* s) {
    kfo_gemv(m, n, A, lda, p, 1.0, 0.0, 0, q);
    kfo_gemvt(m, n, A, lda, r, 1.0, 0.0, 0, s);
}

/* GEMVER (Table 1), A is n x n:
 *   B = A + u1 v1^T + u2 v2^T
 *   x = beta * B^T y + z
 *   w = alpha * B x
 * B is kept in double; x uses the updated B and w the double x. */
void kfo_gemver(int64_t n, const double* A, int64_t lda, const double* u1,
                const double* v1, const double* u2, const double* v2,
                const double* y, const double* z, double alpha, double beta,
                double* B, double* x, double* w) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            B[i * n + j] = A[i * lda + j] + u1[i] * v1[j] + u2[i] * v2[j];
    kfo_gemvt(n, n, B, n, y, beta, 1.0, z, x);
    kfo_gemv(n, n, B, n, x, alpha, 0.0, 0, w);
}

/* GESUMMV (Table 1): y = alpha * A x + beta * B x, A and B m x n. */
void kfo_gesummv(int64_t m, int64_t n, const double* A, const double* B,
                 int64_t lda, const double* x, double alpha, double beta,
                 double* y) {
    for (int64_t i = 0; i < m; ++i) {
        double a = 0.0, b = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            a += A[i * lda + j] * x[j];
            b += B[i * lda + j] * x[j];
        }
        y[i] = alpha * a + beta * b;
    }
}

/* ATAX (Table 1): y = A^T (A x).  t = A x is an internal double vector
 * (workspace of m doubles supplied by the caller). */
void kfo_atax(int64_t m, int64_t n, const double* A, int64_t lda,
              const double* x, double* t, double* y) {
    kfo_gemv(m, n, A, lda, x, 1.0, 0.0, 0, t);
    kfo_gemvt(m, n, A, lda, t, 1.0, 0.0, 0, y);
}

/* AXPYDOT (Table 1): z = w - alpha v ; r = z^T u (z kept in double). */
double kfo_axpydot(int64_t n, const double* w, const double* v,
                   const double* u, double alpha, double* z) {
    kfo_axpby(n, 1.0, w, -alpha, v, z);
    return kfo_dot(n, z, u);
}

/* WAXPBY (Table 1): w = alpha x + beta y. */
void kfo_waxpby(int64_t n, double alpha, const double* x, double beta,
                const double* y, double* w) {
    kfo_axpby(n, alpha, x, beta, y, w);
}

/* Sum of |terms| scales used by the tolerance checks (the usual backward
 * error scale of a dot product): out_i = sum_j |A_ij| |x_j|. */
void kfo_abs_gemv(int64_t m, int64_t n, const double* A, int64_t lda,
                  const double* x, double* out) {
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) acc += fabs(A[i * lda + j]) * fabs(x[j]);
        out[i] = acc;
    }
}

void kfo_abs_gemvt(int64_t m, int64_t n, const double* A, int64_t lda,
                   const double* y, double* out) {
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t i = 0; i < m; ++i) acc += fabs(A[i * lda + j]) * fabs(y[i]);
        out[j] = acc;
    }
}

/* ---------------- Row-scaled low-precision storage of A ----------------
 * The paper is FP32 only (Section 4.1); this storage form is an extension.
 * Reading used (stated, not in the paper): per row i,
 *   s_i = fl32(amax_i / QMAX)   (QMAX = 448 for E4M3, 1 for BF16; s_i = 1
 *                                 when the row is all zero),
 *   Q_ij = round-to-nearest-even into the format of fl32(A_ij / s_i),
 *          saturating to +-448 for E4M3 (no infinities),
 * and the dequantised value is s_i * Q_ij, exact in double.
 * Division here is IEEE single precision division (correctly rounded). */

/* Round a finite float to the nearest bfloat16 (ties to even): keep the top
 * 16 bits of the IEEE-754 single after adding half an ulp of the bf16
 * result plus the tie-break bit. */
static uint16_t f32_to_bf16_rne(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

static double bf16_to_double(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* E4M3 ("fn" variant: no infinities, one NaN pattern): 1 sign bit, 4 exponent
 * bits with bias 7, 3 mantissa bits; largest finite 448 = 1.75 * 2^8;
 * smallest normal 2^-6; subnormals k * 2^-9, k = 1..7.
 * Rounds x to the nearest representable value, ties to even (rint in the
 * default rounding mode), saturating to +-448. */
static uint8_t f32_to_e4m3_rne_sat(float xf) {
    double x = (double)xf;
    uint8_t sign = 0;
    if (x < 0) { sign = 0x80; x = -x; }
    if (x >= 448.0) return (uint8_t)(sign | 0x7E);          /* saturate */
    if (x < ldexp(1.0, -6)) {                                 /* subnormal range */
        double k = rint(x / ldexp(1.0, -9));                  /* 0..8 */
        if (k >= 8.0) return (uint8_t)(sign | 0x08);          /* rounds up to 2^-6 */
        return (uint8_t)(sign | (uint8_t)k);
    }
    int e;
    (void)frexp(x, &e);                /* x = fr * 2^e, fr in [0.5, 1) */
    int E = e - 1;                     /* x = 1.f * 2^E, E in [-6, 8] */
    double quantum = ldexp(1.0, E - 3);
    double q = rint(x / quantum) * quantum;
    if (q >= 448.0) return (uint8_t)(sign | 0x7E);
    /* q may have rounded up to 2^(E+1): re-derive exponent and mantissa */
    (void)frexp(q, &e);
    E = e - 1;
    int mant = (int)rint((q / ldexp(1.0, E) - 1.0) * 8.0);   /* 0..7 */
    int ebits = E + 7;
    return (uint8_t)(sign | (uint8_t)(ebits << 3) | (uint8_t)mant);
}

static double e4m3_to_double(uint8_t b) {
    int sign = b & 0x80;
    int ebits = (b >> 3) & 0xF;
    int mant = b & 0x7;
    double v;
    if (ebits == 0) v = ldexp((double)mant, -9);
    else v = ldexp(1.0 + mant / 8.0, ebits - 7);
    return sign ? -v : v;
}

/* fmt 1 = BF16 (codes: uint16 per element), fmt 2 = E4M3 (uint8 per element).
 * A is FP32 (float*), m x n with leading dimension lda. */
void kfo_quantize_rows(int64_t m, int64_t n, const float* A, int64_t lda,
                       int fmt, void* codes, float* scale) {
    const float qmax = (fmt == 2) ? 448.0f : 1.0f;
    for (int64_t i = 0; i < m; ++i) {
        float amax = 0.0f;
        for (int64_t j = 0; j < n; ++j) {
            float a = fabsf(A[i * lda + j]);
            if (a > amax) amax = a;
        }
        float s = (amax > 0.0f) ? amax / qmax : 1.0f;
        scale[i] = s;
        for (int64_t j = 0; j < n; ++j) {
            float t = A[i * lda + j] / s;
            if (fmt == 2) ((uint8_t*)codes)[i * n + j] = f32_to_e4m3_rne_sat(t);
            else ((uint16_t*)codes)[i * n + j] = f32_to_bf16_rne(t);
        }
    }
}

/* Dequantised matrix Ahat_ij = s_i * Q_ij in double (exact). */
void kfo_dequantize_rows(int64_t m, int64_t n, const void* codes, int fmt,
                         const float* scale, double* Ahat) {
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double q = (fmt == 2) ? e4m3_to_double(((const uint8_t*)codes)[i * n + j])
                                  : bf16_to_double(((const uint16_t*)codes)[i * n + j]);
            Ahat[i * n + j] = (double)scale[i] * q;
        }
}

/* Element decoders exposed for the pins. */
double kfo_bf16_value(uint16_t h) { return bf16_to_double(h); }
double kfo_e4m3_value(uint8_t b) { return e4m3_to_double(b); }
uint16_t kfo_bf16_code(float f) { return f32_to_bf16_rne(f); }
uint8_t kfo_e4m3_code(float f) { return f32_to_e4m3_rne_sat(f); }

/* GEMVER with row-scaled storage (the library's low-precision GEMVER; the
 * paper is FP32 only).  A is given as codes QA with row scales sA.  The
 * storage rule of B = Ahat + u1 v1^T + u2 v2^T, whose codes are integer
 * decisions taken in FP32 (the precision the rule is stated in):
 *   sB_i  = (sA_i * QMAX + |u1_i| max_j |v1_j| + |u2_i| max_j |v2_j|) / QMAX,
 *           left to right, 1 when the bound is 0 (QMAX = 1 BF16, 448 E4M3);
 *   b_ij  = fma(u2_i, v2_j, fma(u1_i, v1_j, sA_i * QA_ij));
 *   QB_ij = round-to-nearest-even of b_ij * (1 / sB_i) (E4M3 saturating).
 * Writes QB (n x n codes, row length n) and sB.  x and w follow in double
 * from the stored matrix (kfo_dequantize_rows, kfo_gemvt, kfo_gemv). */
void kfo_gemver_rowscaled_store(int64_t n, const void* qa, int fmt, const float* sa,
                                const float* u1, const float* v1, const float* u2,
                                const float* v2, void* qb, float* sb) {
    const float qmax = (fmt == 2) ? 448.0f : 1.0f;
    float n1 = 0.0f, n2 = 0.0f;
    for (int64_t j = 0; j < n; ++j) {
        if (fabsf(v1[j]) > n1) n1 = fabsf(v1[j]);
        if (fabsf(v2[j]) > n2) n2 = fabsf(v2[j]);
    }
    for (int64_t i = 0; i < n; ++i) {
        float bound = sa[i] * qmax;
        bound = bound + fabsf(u1[i]) * n1;
        bound = bound + fabsf(u2[i]) * n2;
        const float s = (bound > 0.0f) ? bound / qmax : 1.0f;
        const float inv = 1.0f / s;
        sb[i] = s;
        for (int64_t j = 0; j < n; ++j) {
            const float q = (fmt == 2) ? (float)e4m3_to_double(((const uint8_t*)qa)[i * n + j])
                                       : (float)bf16_to_double(((const uint16_t*)qa)[i * n + j]);
            const float a = sa[i] * q;
            const float b = fmaf(u2[i], v2[j], fmaf(u1[i], v1[j], a));
            const float t = b * inv;
            if (fmt == 2) ((uint8_t*)qb)[i * n + j] = f32_to_e4m3_rne_sat(t);
            else ((uint16_t*)qb)[i * n + j] = f32_to_bf16_rne(t);
        }
    }
}
