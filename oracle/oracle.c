/*
 * FP64 CPU oracle for the GA-offload loop program.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: it is used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference leg of bench.py.  It shares no code, header or
 * constant table with the CUDA library (paper_1806_01430_gb300/csrc).
 *
 * What it computes.  The paper (Sec. 4, Sec. 5.1.1) offloads the `for` loops of a
 * matrix-manipulation program and states that a gene only moves loops between
 * CPU and GPU; the program's result does not depend on the gene.  The oracle is
 * therefore the plain definition of each loop of the program, evaluated in
 * program order in IEEE double precision:
 *
 *   INIT       x = u24 * 2^-23 - 1, u24 a 24-bit field of h = SplitMix64(key)  [input generator]
 *   GEMM       C = alpha * A B + beta * C0          (Sec. 5.1.1: matrix product benchmark)
 *   AXPY       D = X + alpha * Y                    (scale-add, D = C + 2A)
 *   TRANSPOSE  E = D^T
 *   ROWSUM     r_i = sum_j E_ij
 *   FROBENIUS  f = sqrt(sum_ij E_ij^2)
 *   RELU       F = max(E, 0)
 *   SQUARE     H = G (.) G
 *   COLMAX     q_j = max_i P_ij
 *   SUM        s = sum_ij P_ij
 *   STENCIL3   Y_ij = sum_{a,b in -1..1} w_ab X_{i+a, j+b}, X = 0 outside the image
 *              (image-analysis loops, the paper's motivating IoT camera workload, Sec. 1)
 *   RECURRENCE Y_i0 = X_i0, Y_ij = alpha Y_i,j-1 + X_ij   (a loop-carried dependence)
 *   FIND       k_i = min { j : X_ij > t } (cols if none), t = alpha rounded to binary32
 *              (a loop with an early exit); both are loops Sec. 4 keeps on the CPU
 *
 * Every loop is the textbook double/triple loop.  The GEMM runs its loops in
 * i-k-j order so that the row of B is read contiguously; for every output
 * element the sum over k is still taken in ascending k, exactly the definition.
 *
 * The counter hash (SplitMix64, Steele, Lea & Flood, OOPSLA 2014) is written here
 * from its published definition; the CUDA library has its own copy, written
 * separately from the same definition.  Seeded inputs are therefore identical
 * on both sides without either side calling the other.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- SplitMix64 -------------------------------------------------------- */
/* The generator's state advances by the odd constant gamma = 0x9E3779B97F4A7C15;
 * each output is the state passed through the published 64-bit finaliser
 * (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31). */
#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t orc_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* First output of a SplitMix64 generator whose state is `state`. */
uint64_t orc_splitmix64(uint64_t state) { return orc_finalise(state + ORC_GAMMA); }

/* n consecutive outputs of one generator seeded with `seed` (test-vector helper). */
void orc_splitmix64_stream(uint64_t seed, int64_t n, uint64_t *out) {
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) {
        s += ORC_GAMMA;
        out[i] = orc_finalise(s);
    }
}

/* Key of element `idx` of buffer `buf` for a program seeded with `seed`:
 * seed in bits 40.., buffer id in bits 36..39, element index in bits 0..35. */
static uint64_t orc_key(uint64_t seed, uint64_t buf, uint64_t idx) {
    return (seed << 40) ^ (buf << 36) ^ idx;
}

/* U[-1,1) value of element idx of buffer buf: a 24-bit integer scaled by 2^-23,
 * minus one, exactly representable in binary32.  One hash serves two elements:
 * element 2j takes bits 40..63 and element 2j+1 bits 16..39 of the hash of key j. */
double orc_init_value(uint64_t seed, int64_t buf, int64_t idx) {
    uint64_t h = orc_splitmix64(orc_key(seed, (uint64_t)buf, (uint64_t)(idx >> 1)));
    int64_t u24 = (idx & 1) ? (int64_t)((h >> 16) & 0xFFFFFFu) : (int64_t)(h >> 40);
    return (double)(u24 - (1LL << 23)) / 8388608.0;
}

static int64_t orc_floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* Power-of-two exponent of the row factor used for the row-scaled input set:
 * z = (sum of 12 U[0,1) draws) - 6  (Irwin-Hall approximation of N(0,1)),
 * e = round(z * 10/3) clamped to [-10, 10], so the factor 2^e spans about
 * 1e-3 .. 1e3 at +-3 sigma.  Draws come from buffer id 15, element row*12+t.
 * Computed in integers so that it is exact. */
int64_t orc_row_exponent(uint64_t seed, int64_t row) {
    int64_t s = 0;
    for (int t = 0; t < 12; ++t) {
        uint64_t h = orc_splitmix64(orc_key(seed, 15u, (uint64_t)(row * 12 + t)));
        s += (int64_t)(h >> 40);
    }
    const int64_t two24 = 1LL << 24;
    int64_t num = (s - 6 * two24) * 10; /* z * 10 * 2^24 */
    int64_t den = 3 * two24;            /* 3 * 2^24 */
    int64_t e = orc_floor_div(2 * num + den, 2 * den); /* round half up of num/den */
    if (e < -10) e = -10;
    if (e > 10) e = 10;
    return e;
}

/* INIT loop: out[i][j] = value(seed, buf, i*cols + j) (times 2^e_i if rowscale). */
void orc_init(uint64_t seed, int64_t buf, int64_t rows, int64_t cols, int rowscale, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i) {
        double f = rowscale ? ldexp(1.0, (int)orc_row_exponent(seed, i)) : 1.0;
        for (int64_t j = 0; j < cols; ++j) out[i * cols + j] = orc_init_value(seed, buf, i * cols + j) * f;
    }
}

/* GEMM loop: C[i][j] = alpha * sum_k A[i][k] B[k][j] + beta * C0[i][j].
 * A is M x K, B is K x N, C0 and C are M x N, all row-major.  C0 may equal C. */
void orc_gemm(int64_t M, int64_t N, int64_t K, double alpha, const double *A, const double *B,
              double beta, const double *C0, double *C) {
#pragma omp parallel
    {
        /* per-thread row accumulator */
        double *acc = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < M; ++i) {
            for (int64_t j = 0; j < N; ++j) acc[j] = 0.0;
            for (int64_t k = 0; k < K; ++k) {
                const double a = A[i * K + k];
                const double *brow = B + k * N;
                for (int64_t j = 0; j < N; ++j) acc[j] += a * brow[j];
            }
            for (int64_t j = 0; j < N; ++j) C[i * N + j] = alpha * acc[j] + beta * C0[i * N + j];
        }
        free(acc);
    }
}

/* AXPY loop: out = x + alpha * y, elementwise over n entries. */
void orc_axpy(int64_t n, const double *x, double alpha, const double *y, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = x[i] + alpha * y[i];
}

/* TRANSPOSE loop: out (cols x rows) = in (rows x cols)^T. */
void orc_transpose(int64_t rows, int64_t cols, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) out[j * rows + i] = in[i * cols + j];
}

/* ROWSUM loop: out[i] = sum_j in[i][j]. */
void orc_rowsum(int64_t rows, int64_t cols, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < cols; ++j) s += in[i * cols + j];
        out[i] = s;
    }
}

/* FROBENIUS loop: sqrt(sum of squares), summed in index order. */
double orc_frobenius(int64_t n, const double *in) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += in[i] * in[i];
    return sqrt(s);
}

/* RELU loop: out = max(in, 0). */
void orc_relu(int64_t n, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = in[i] > 0.0 ? in[i] : 0.0;
}

/* SQUARE loop: out = in (.) in. */
void orc_square(int64_t n, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = in[i] * in[i];
}

/* COLMAX loop: out[j] = max_i in[i][j]. */
void orc_colmax(int64_t rows, int64_t cols, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < cols; ++j) {
        double m = -INFINITY;
        for (int64_t i = 0; i < rows; ++i)
            if (in[i * cols + j] > m) m = in[i * cols + j];
        out[j] = m;
    }
}

/* SUM loop: sum of all entries in index order. */
double orc_sum(int64_t n, const double *in) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += in[i];
    return s;
}

/* Weights of the 3x3 stencil presets, row-major over (a, b) = (-1..1, -1..1):
 * 0 binomial blur (1 2 1; 2 4 2; 1 2 1) / 16, 1 Laplacian (0 1 0; 1 -4 1; 0 1 0),
 * 2 Sobel x (-1 0 1; -2 0 2; -1 0 1), 3 Sobel y (-1 -2 -1; 0 0 0; 1 2 1). */
static const double ORC_STENCIL_W[4][9] = {
    {1.0 / 16, 2.0 / 16, 1.0 / 16, 2.0 / 16, 4.0 / 16, 2.0 / 16, 1.0 / 16, 2.0 / 16, 1.0 / 16},
    {0, 1, 0, 1, -4, 1, 0, 1, 0},
    {-1, 0, 1, -2, 0, 2, -1, 0, 1},
    {-1, -2, -1, 0, 0, 0, 1, 2, 1},
};

/* STENCIL3 loop: out[i][j] = sum of w[a][b] * in[i+a][j+b] over a, b in {-1, 0, 1},
 * terms outside the image taken as 0. */
int orc_stencil3(int64_t rows, int64_t cols, const double *in, int preset, double *out) {
    if (preset < 0 || preset > 3) return -1;
    const double *w = ORC_STENCIL_W[preset];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            double s = 0.0;
            for (int a = -1; a <= 1; ++a)
                for (int b = -1; b <= 1; ++b) {
                    const int64_t y = i + a, x = j + b;
                    if (y >= 0 && y < rows && x >= 0 && x < cols) s += w[(a + 1) * 3 + (b + 1)] * in[y * cols + x];
                }
            out[i * cols + j] = s;
        }
    return 0;
}

/* RECURRENCE loop along each row, in binary64. */
void orc_recurrence(int64_t rows, int64_t cols, const double *in, double alpha, double *out) {
    for (int64_t i = 0; i < rows; ++i) {
        const double *x = in + i * cols;
        double *y = out + i * cols;
        for (int64_t j = 0; j < cols; ++j) y[j] = j == 0 ? x[0] : alpha * y[j - 1] + x[j];
    }
}

/* FIND loop: the first column whose element exceeds the threshold (the threshold is the
 * binary32 value of alpha, the precision the loop's data has). */
void orc_find(int64_t rows, int64_t cols, const double *in, double alpha, double *out) {
    const double t = (double)(float)alpha;
    for (int64_t i = 0; i < rows; ++i) {
        int64_t k = cols;
        for (int64_t j = cols - 1; j >= 0; --j)
            if (in[i * cols + j] > t) k = j;
        out[i] = (double)k;
    }
}

/* ---- sampled entries at full size, without materialising the matrices ---- */

/* C[i][j] of the GEMM loop applied to freshly initialised A (buffer bufA, M x K,
 * optionally row-scaled), B (bufB, K x N) and C0 (bufC, M x N), for the listed
 * (i, j) pairs.  Lets tests check full-size runs entry by entry. */
void orc_gemm_init_entries(uint64_t seed, int64_t bufA, int64_t bufB, int64_t bufC, int rowscaleA,
                           int64_t M, int64_t N, int64_t K, double alpha, double beta, int64_t n_samples,
                           const int64_t *ii, const int64_t *jj, double *out) {
    (void)M;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_samples; ++s) {
        const int64_t i = ii[s], j = jj[s];
        const double f = rowscaleA ? ldexp(1.0, (int)orc_row_exponent(seed, i)) : 1.0;
        double acc = 0.0;
        for (int64_t k = 0; k < K; ++k)
            acc += (orc_init_value(seed, bufA, i * K + k) * f) * orc_init_value(seed, bufB, k * N + j);
        out[s] = alpha * acc + beta * orc_init_value(seed, bufC, i * N + j);
    }
}

/* Column `j` of the GEMM output (all M rows) computed from given A, B, C0 in double;
 * used for full-size row-sum checks.  A is M x K, B is K x N (row-major). */
void orc_gemm_column(int64_t M, int64_t N, int64_t K, double alpha, const double *A, const double *B,
                     double beta, const double *C0, int64_t j, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        double acc = 0.0;
        for (int64_t k = 0; k < K; ++k) acc += A[i * K + k] * B[k * N + j];
        out[i] = alpha * acc + beta * C0[i * N + j];
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
