/*
 * CPU oracle for the annotated-launch hot path (test infrastructure only).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header or constant table with the
 * CUDA path: every function below is the plain, unchunked, sequential
 * definition of what a workload computes.  The method guarantees that
 * chunked, asynchronous execution reaches exactly this result (sequential
 * consistency, Sec. 1 and Sec. 2.4 "Execution Planner": distributions
 * affect performance, not correctness).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fast-math, so
 * every f32/f64 operation is a single IEEE-754 round-to-nearest operation).
 * OpenMP only splits independent rows, samples or array slices; it never
 * changes an arithmetic order.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Seeded inputs: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), written    */
/* from its published definition, evaluated by counter.                      */
/* ------------------------------------------------------------------------ */
#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_next(uint64_t *state) {
    *state += ORC_GAMMA;
    return orc_mix64(*state);
}

uint64_t orc_stream_key(uint64_t seed, uint64_t stream) {
    uint64_t s = seed ^ (stream << 32);
    return orc_splitmix64_next(&s);
}

static inline uint64_t orc_elem(uint64_t key, uint64_t idx) {
    return orc_mix64(key + (idx + 1) * ORC_GAMMA);
}

static inline float orc_u01_f32(uint64_t x) { return (float)(x >> 40) * 0x1p-24f; }

void orc_gen_u64(uint64_t seed, uint64_t stream, uint64_t idx0, int64_t n, uint64_t *out) {
    uint64_t key = orc_stream_key(seed, stream);
    for (int64_t k = 0; k < n; ++k) out[k] = orc_elem(key, idx0 + (uint64_t)k);
}

void orc_gen_uniform_f32(uint64_t seed, uint64_t stream, uint64_t idx0, int64_t n, float *out) {
    uint64_t key = orc_stream_key(seed, stream);
#pragma omp parallel for schedule(static) if (n > (1 << 20))
    for (int64_t k = 0; k < n; ++k) out[k] = orc_u01_f32(orc_elem(key, idx0 + (uint64_t)k));
}

void orc_gen_u8(uint64_t seed, uint64_t stream, uint64_t idx0, int64_t n, uint8_t *out) {
    uint64_t key = orc_stream_key(seed, stream);
#pragma omp parallel for schedule(static) if (n > (1 << 20))
    for (int64_t k = 0; k < n; ++k) out[k] = (uint8_t)(orc_elem(key, idx0 + (uint64_t)k) >> 56);
}

static inline float orc_kappa_of(uint64_t x) {
    double u = (double)orc_u01_f32(x);
    return (float)(0.05 + 0.15 * u);
}

void orc_gen_kappa_f32(uint64_t seed, uint64_t stream, uint64_t idx0, int64_t n, float *out) {
    uint64_t key = orc_stream_key(seed, stream);
    for (int64_t k = 0; k < n; ++k) out[k] = orc_kappa_of(orc_elem(key, idx0 + (uint64_t)k));
}

/* round-to-nearest-even of an f32 bit pattern to bf16 (finite inputs) */
static inline uint16_t orc_f32_to_bf16(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    uint32_t lsb = (b >> 16) & 1u;
    return (uint16_t)((b + 0x7FFFu + lsb) >> 16);
}

static inline double orc_bf16_to_f64(uint16_t h) {
    uint32_t b = (uint32_t)h << 16;
    float f;
    memcpy(&f, &b, 4);
    return (double)f;
}

/* N(0,1)*scale by Box-Muller from counters 2*idx and 2*idx+1; returns the
 * unrounded fp64 value, *bits receives its f32-then-bf16 RNE rounding. */
static inline double orc_normal(uint64_t key, uint64_t idx, double scale, uint16_t *bits) {
    uint64_t x1 = orc_elem(key, 2 * idx), x2 = orc_elem(key, 2 * idx + 1);
    double u1 = ((double)(x1 >> 11) + 1.0) * 0x1p-53;
    double u2 = (double)(x2 >> 11) * 0x1p-53;
    double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    double v = z * scale;
    *bits = orc_f32_to_bf16((float)v);
    return v;
}

void orc_gen_normal_bf16(uint64_t seed, uint64_t stream, uint64_t idx0, int64_t n, double scale,
                         uint16_t *bits) {
    uint64_t key = orc_stream_key(seed, stream);
#pragma omp parallel for schedule(static) if (n > (1 << 18))
    for (int64_t k = 0; k < n; ++k) orc_normal(key, idx0 + (uint64_t)k, scale, &bits[k]);
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Worked example of the paper (Listings 1-2, host code of Sec. 3.6):       */
/* out[i] = (in[i-1] + in[i] + in[i+1]) / 3.0, out-of-range reads give 0.   */
/* The sum is in float; "/ 3.0" is a double literal, so the division runs   */
/* in double and the store rounds back to float.                             */
/* ------------------------------------------------------------------------ */
void orc_stencil1d_paper(int64_t n, const float *in, float *out) {
    for (int64_t i = 0; i < n; ++i) {
        float left = i - 1 >= 0 ? in[i - 1] : 0.0f;
        float mid = in[i];
        float right = i + 1 < n ? in[i + 1] : 0.0f;
        float s = left + mid;
        s = s + right;
        out[i] = (float)((double)s / 3.0);
    }
}

/* ------------------------------------------------------------------------ */
/* 2-D 5-point Jacobi (the HotSpot-like stencil of Sec. 4.2), f32:          */
/*   V[i,j] = ((((U[i,j] + U[i-1,j]) + U[i+1,j]) + U[i,j-1]) + U[i,j+1]) / 5 */
/* reads outside the domain give 0 (the listings' "? ... : 0" ghosts).      */
/* ------------------------------------------------------------------------ */
static void orc_jacobi2d_f32_step(int64_t ny, int64_t nx, const float *u, float *v) {
#pragma omp parallel for schedule(static) if (ny * nx > (1 << 16))
    for (int64_t i = 0; i < ny; ++i) {
        for (int64_t j = 0; j < nx; ++j) {
            float c = u[i * nx + j];
            float n = i > 0 ? u[(i - 1) * nx + j] : 0.0f;
            float s = i + 1 < ny ? u[(i + 1) * nx + j] : 0.0f;
            float w = j > 0 ? u[i * nx + j - 1] : 0.0f;
            float e = j + 1 < nx ? u[i * nx + j + 1] : 0.0f;
            float acc = c + n;
            acc = acc + s;
            acc = acc + w;
            acc = acc + e;
            v[i * nx + j] = acc / 5.0f;
        }
    }
}

/* iters steps from in; result in out (in and out may alias); 0 on success */
int orc_jacobi2d_f32(int64_t ny, int64_t nx, const float *in, float *out, int iters) {
    size_t bytes = (size_t)(ny * nx) * sizeof(float);
    float *a = (float *)malloc(bytes), *b = (float *)malloc(bytes);
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, in, bytes);
    for (int t = 0; t < iters; ++t) {
        orc_jacobi2d_f32_step(ny, nx, a, b);
        float *tmp = a; a = b; b = tmp;
    }
    memcpy(out, a, bytes);
    free(a);
    free(b);
    return 0;
}

/* Same update in f64 on an (ny+2) x (nx+2) array whose outer ring holds the
 * ghost values (kept fixed), or, if periodic != 0, is refreshed from the
 * opposite edges before every step.  Used only to pin the definition. */
int orc_jacobi2d_f64_ring(int64_t ny, int64_t nx, double *p, int iters, int periodic) {
    int64_t W = nx + 2;
    size_t bytes = (size_t)((ny + 2) * W) * sizeof(double);
    double *q = (double *)malloc(bytes);
    if (!q) return -1;
    for (int t = 0; t < iters; ++t) {
        if (periodic) {
            for (int64_t j = 1; j <= nx; ++j) {
                p[0 * W + j] = p[ny * W + j];
                p[(ny + 1) * W + j] = p[1 * W + j];
            }
            for (int64_t i = 1; i <= ny; ++i) {
                p[i * W + 0] = p[i * W + nx];
                p[i * W + nx + 1] = p[i * W + 1];
            }
        }
        memcpy(q, p, bytes);
        for (int64_t i = 1; i <= ny; ++i)
            for (int64_t j = 1; j <= nx; ++j) {
                double acc = p[i * W + j] + p[(i - 1) * W + j];
                acc = acc + p[(i + 1) * W + j];
                acc = acc + p[i * W + j - 1];
                acc = acc + p[i * W + j + 1];
                q[i * W + j] = acc / 5.0;
            }
        memcpy(p, q, bytes);
    }
    free(q);
    return 0;
}

/* Value of sampled cells of the f32 Jacobi after `iters` steps on an
 * NY x NX field whose initial values are the seeded uniform stream.  A cell
 * after T steps depends only on initial cells within distance T, so each
 * sample runs the plain f32 Jacobi on the (2T+1)^2 window around it (clipped
 * to the domain); window cells outside the domain are true zero ghosts,
 * other window-edge errors move one cell per step and never reach the
 * centre. */
int orc_jacobi2d_f32_lightcone(int64_t NY, int64_t NX, uint64_t seed, uint64_t stream, int iters,
                               int64_t nsamp, const int64_t *si, const int64_t *sj, float *out) {
    int failed = 0;
    uint64_t key = orc_stream_key(seed, stream);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
    for (int64_t s = 0; s < nsamp; ++s) {
        int64_t r0 = si[s] - iters < 0 ? 0 : si[s] - iters;
        int64_t r1 = si[s] + iters > NY - 1 ? NY - 1 : si[s] + iters;
        int64_t c0 = sj[s] - iters < 0 ? 0 : sj[s] - iters;
        int64_t c1 = sj[s] + iters > NX - 1 ? NX - 1 : sj[s] + iters;
        int64_t h = r1 - r0 + 1, w = c1 - c0 + 1;
        float *win = (float *)malloc((size_t)(h * w) * sizeof(float));
        if (!win) { failed |= 1; continue; }
        for (int64_t r = 0; r < h; ++r)
            for (int64_t c = 0; c < w; ++c)
                win[r * w + c] = orc_u01_f32(orc_elem(key, (uint64_t)((r0 + r) * NX + (c0 + c))));
        /* clipped rows/cols at the domain edge are exact; interior window
         * edges are at distance >= iters from the centre */
        float *a = win, *b = (float *)malloc((size_t)(h * w) * sizeof(float));
        if (!b) { free(win); failed |= 1; continue; }
        for (int t = 0; t < iters; ++t) {
            for (int64_t i = 0; i < h; ++i)
                for (int64_t j = 0; j < w; ++j) {
                    float c = a[i * w + j];
                    float n = i > 0 ? a[(i - 1) * w + j] : 0.0f;
                    float so = i + 1 < h ? a[(i + 1) * w + j] : 0.0f;
                    float we = j > 0 ? a[i * w + j - 1] : 0.0f;
                    float e = j + 1 < w ? a[i * w + j + 1] : 0.0f;
                    float acc = c + n;
                    acc = acc + so;
                    acc = acc + we;
                    acc = acc + e;
                    b[i * w + j] = acc / 5.0f;
                }
            float *tmp = a; a = b; b = tmp;
        }
        out[s] = a[(si[s] - r0) * w + (sj[s] - c0)];
        free(a);
        free(b);
    }
    return failed ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* 3-D 7-point Jacobi, f32, zero ghosts, summation order                    */
/* centre, z-1, z+1, y-1, y+1, x-1, x+1, then / 7.                           */
/* ------------------------------------------------------------------------ */
int orc_jacobi3d_f32(int64_t nz, int64_t ny, int64_t nx, const float *in, float *out, int iters) {
    size_t n = (size_t)(nz * ny * nx);
    float *a = (float *)malloc(n * sizeof(float)), *b = (float *)malloc(n * sizeof(float));
    if (!a || !b) { free(a); free(b); return -1; }
    memcpy(a, in, n * sizeof(float));
    for (int t = 0; t < iters; ++t) {
#pragma omp parallel for schedule(static) if (n > (1 << 16))
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    int64_t o = (z * ny + y) * nx + x;
                    float acc = a[o];
                    acc = acc + (z > 0 ? a[o - ny * nx] : 0.0f);
                    acc = acc + (z + 1 < nz ? a[o + ny * nx] : 0.0f);
                    acc = acc + (y > 0 ? a[o - nx] : 0.0f);
                    acc = acc + (y + 1 < ny ? a[o + nx] : 0.0f);
                    acc = acc + (x > 0 ? a[o - 1] : 0.0f);
                    acc = acc + (x + 1 < nx ? a[o + 1] : 0.0f);
                    b[o] = acc / 7.0f;
                }
        float *tmp = a; a = b; b = tmp;
    }
    memcpy(out, a, n * sizeof(float));
    free(a);
    free(b);
    return 0;
}

/* f64 twin with zero ghosts, used only for the closed-form pin */
int orc_jacobi3d_f64(int64_t nz, int64_t ny, int64_t nx, double *u, int iters) {
    size_t n = (size_t)(nz * ny * nx);
    double *b = (double *)malloc(n * sizeof(double));
    if (!b) return -1;
    for (int t = 0; t < iters; ++t) {
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    int64_t o = (z * ny + y) * nx + x;
                    double acc = u[o];
                    acc = acc + (z > 0 ? u[o - ny * nx] : 0.0);
                    acc = acc + (z + 1 < nz ? u[o + ny * nx] : 0.0);
                    acc = acc + (y > 0 ? u[o - nx] : 0.0);
                    acc = acc + (y + 1 < ny ? u[o + nx] : 0.0);
                    acc = acc + (x > 0 ? u[o - 1] : 0.0);
                    acc = acc + (x + 1 < nx ? u[o + 1] : 0.0);
                    b[o] = acc / 7.0;
                }
        memcpy(u, b, n * sizeof(double));
    }
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* GEMM C = A B (Sec. 4.2 "GEMM"): plain fp64 triple loop, k ascending.     */
/* ------------------------------------------------------------------------ */
void orc_gemm_f64(int64_t M, int64_t N, int64_t K, const double *A, const double *B, double *C) {
#pragma omp parallel for schedule(static) if (M * N * K > (1 << 22))
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = 0; j < N; ++j) {
            double acc = 0.0;
            for (int64_t k = 0; k < K; ++k) acc += A[i * K + k] * B[k * N + j];
            C[i * N + j] = acc;
        }
}

/* Entries C[rows[r], cols[c]] of C = A B where A (M x K) and B (K x N) are
 * the seeded N(0,1)*scale streams (A[i,k] at index i*K+k of streamA, B[k,j]
 * at index k*N+j of streamB).  C_rounded uses the bf16-rounded inputs
 * (exactly representable in fp64), C_unrounded the fp64 values before
 * rounding.  Output is nr x nc row-major. */
int orc_gemm_sample_f64(int64_t M, int64_t N, int64_t K, uint64_t seed, uint64_t streamA,
                        uint64_t streamB, double scale, int64_t nr, const int64_t *rows, int64_t nc,
                        const int64_t *cols, double *C_rounded, double *C_unrounded) {
    (void)M;
    uint64_t ka = orc_stream_key(seed, streamA), kb = orc_stream_key(seed, streamB);
    double *ar = (double *)malloc((size_t)(nr * K) * sizeof(double));
    double *au = (double *)malloc((size_t)(nr * K) * sizeof(double));
    double *br = (double *)malloc((size_t)(nc * K) * sizeof(double));
    double *bu = (double *)malloc((size_t)(nc * K) * sizeof(double));
    if (!ar || !au || !br || !bu) { free(ar); free(au); free(br); free(bu); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nr; ++r)
        for (int64_t k = 0; k < K; ++k) {
            uint16_t bits;
            au[r * K + k] = orc_normal(ka, (uint64_t)(rows[r] * K + k), scale, &bits);
            ar[r * K + k] = orc_bf16_to_f64(bits);
        }
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c)
        for (int64_t k = 0; k < K; ++k) {
            uint16_t bits;
            bu[c * K + k] = orc_normal(kb, (uint64_t)(k * N + cols[c]), scale, &bits);
            br[c * K + k] = orc_bf16_to_f64(bits);
        }
#pragma omp parallel for schedule(static) collapse(2)
    for (int64_t r = 0; r < nr; ++r)
        for (int64_t c = 0; c < nc; ++c) {
            double s1 = 0.0, s2 = 0.0;
            for (int64_t k = 0; k < K; ++k) {
                s1 += ar[r * K + k] * br[c * K + k];
                s2 += au[r * K + k] * bu[c * K + k];
            }
            C_rounded[r * nc + c] = s1;
            C_unrounded[r * nc + c] = s2;
        }
    free(ar); free(au); free(br); free(bu);
    return 0;
}

/* f32 GEMM of the seeded bf16 inputs over an M x N x K corner (row-major
 * f32 result), plain loop: used only as the timed CPU baseline. */
int orc_gemm_bf16_corner_f32(int64_t M, int64_t N, int64_t K, int64_t ldN, int64_t ldK, uint64_t seed,
                             uint64_t streamA, uint64_t streamB, double scale, float *C) {
    uint64_t ka = orc_stream_key(seed, streamA), kb = orc_stream_key(seed, streamB);
    float *A = (float *)malloc((size_t)(M * K) * sizeof(float));
    float *B = (float *)malloc((size_t)(K * N) * sizeof(float));
    if (!A || !B) { free(A); free(B); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i)
        for (int64_t k = 0; k < K; ++k) {
            uint16_t bits;
            orc_normal(ka, (uint64_t)(i * ldK + k), scale, &bits);
            A[i * K + k] = (float)orc_bf16_to_f64(bits);
        }
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < K; ++k)
        for (int64_t j = 0; j < N; ++j) {
            uint16_t bits;
            orc_normal(kb, (uint64_t)(k * ldN + j), scale, &bits);
            B[k * N + j] = (float)orc_bf16_to_f64(bits);
        }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < N; ++j) C[i * N + j] = 0.0f;
        for (int64_t k = 0; k < K; ++k) {
            float a = A[i * K + k];
            for (int64_t j = 0; j < N; ++j) C[i * N + j] += a * B[k * N + j];
        }
    }
    free(A);
    free(B);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 256-bin histogram, H[b] = #{i : x[i] = b}: the reduce(+) pattern of       */
/* Sec. 2.3 ("reduce(f)").                                                    */
/* ------------------------------------------------------------------------ */
void orc_hist256(int64_t n, const uint8_t *x, uint32_t *h) {
    for (int b = 0; b < 256; ++b) h[b] = 0;
    for (int64_t i = 0; i < n; ++i) h[x[i]] += 1u;
}

/* ------------------------------------------------------------------------ */
/* Row reduction, the paper's third annotation example (Sec. 2.3):          */
/*   "global [i, j] => read A[i, j], reduce(f) sum[i]",  f in {+, *, min, max} */
/* out[i] = A[i,0] f A[i,1] f ... f A[i,nx-1], in fp64, left to right.        */
/* op: 0 = +, 1 = *, 2 = min, 3 = max.                                        */
/* ------------------------------------------------------------------------ */
void orc_rowreduce_f64(int64_t ny, int64_t nx, const double *a, int op, double *out) {
    for (int64_t i = 0; i < ny; ++i) {
        double acc = a[i * nx];
        for (int64_t j = 1; j < nx; ++j) {
            double x = a[i * nx + j];
            if (op == 0)
                acc = acc + x;
            else if (op == 1)
                acc = acc * x;
            else if (op == 2)
                acc = x < acc ? x : acc;
            else
                acc = x > acc ? x : acc;
        }
        out[i] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Variable-coefficient diffusion and its adjoint, fp64:                    */
/*   (L u)_ij = (((u_{i-1,j} + u_{i+1,j}) + u_{i,j-1}) + u_{i,j+1}) - 4 u_ij */
/*   u_{t+1} = u_t + kappa (.) L u_t,   J = sum u_T^2                          */
/*   lambda_T = 2 u_T,  lambda_t = lambda_{t+1} + L(kappa (.) lambda_{t+1})    */
/*   dJ/dkappa = sum_t lambda_{t+1} (.) L u_t,   dJ/du_0 = lambda_0            */
/* zero ghosts outside the domain (L is symmetric, so L^T = L).               */
/* ------------------------------------------------------------------------ */
static void orc_lap_f64(int64_t ny, int64_t nx, const double *u, double *out) {
    for (int64_t i = 0; i < ny; ++i)
        for (int64_t j = 0; j < nx; ++j) {
            double n = i > 0 ? u[(i - 1) * nx + j] : 0.0;
            double s = i + 1 < ny ? u[(i + 1) * nx + j] : 0.0;
            double w = j > 0 ? u[i * nx + j - 1] : 0.0;
            double e = j + 1 < nx ? u[i * nx + j + 1] : 0.0;
            out[i * nx + j] = (((n + s) + w) + e) - 4.0 * u[i * nx + j];
        }
}

int orc_diff_forward_f64(int64_t ny, int64_t nx, const double *u0, const double *kappa, int T,
                         double *uT) {
    size_t n = (size_t)(ny * nx);
    double *u = (double *)malloc(n * sizeof(double)), *l = (double *)malloc(n * sizeof(double));
    if (!u || !l) { free(u); free(l); return -1; }
    memcpy(u, u0, n * sizeof(double));
    for (int t = 0; t < T; ++t) {
        orc_lap_f64(ny, nx, u, l);
        for (size_t k = 0; k < n; ++k) u[k] = u[k] + kappa[k] * l[k];
    }
    memcpy(uT, u, n * sizeof(double));
    free(u);
    free(l);
    return 0;
}

/* J, dJ/du0 and dJ/dkappa; stores every state (plain, no checkpointing) */
int orc_diff_grad_f64(int64_t ny, int64_t nx, const double *u0, const double *kappa, int T, double *J,
                      double *du0, double *dkappa) {
    size_t n = (size_t)(ny * nx);
    double *U = (double *)malloc((size_t)(T + 1) * n * sizeof(double));
    double *l = (double *)malloc(n * sizeof(double));
    double *lam = (double *)malloc(n * sizeof(double));
    double *kl = (double *)malloc(n * sizeof(double));
    if (!U || !l || !lam || !kl) { free(U); free(l); free(lam); free(kl); return -1; }
    memcpy(U, u0, n * sizeof(double));
    for (int t = 0; t < T; ++t) {
        orc_lap_f64(ny, nx, U + (size_t)t * n, l);
        for (size_t k = 0; k < n; ++k) U[(size_t)(t + 1) * n + k] = U[(size_t)t * n + k] + kappa[k] * l[k];
    }
    double j = 0.0;
    const double *uT = U + (size_t)T * n;
    for (size_t k = 0; k < n; ++k) j += uT[k] * uT[k];
    *J = j;
    for (size_t k = 0; k < n; ++k) { lam[k] = 2.0 * uT[k]; dkappa[k] = 0.0; }
    for (int t = T - 1; t >= 0; --t) {
        orc_lap_f64(ny, nx, U + (size_t)t * n, l);
        for (size_t k = 0; k < n; ++k) dkappa[k] += lam[k] * l[k];
        for (size_t k = 0; k < n; ++k) kl[k] = kappa[k] * lam[k];
        orc_lap_f64(ny, nx, kl, l);
        for (size_t k = 0; k < n; ++k) lam[k] = lam[k] + l[k];
    }
    memcpy(du0, lam, n * sizeof(double));
    free(U); free(l); free(lam); free(kl);
    return 0;
}

/* Sampled u_T, dJ/du0 and dJ/dkappa at cells (si, sj) of an NY x NX field
 * whose u0 and kappa are the seeded f32 streams (widened to fp64).  u_T at a
 * cell depends on u0 within distance T, and the gradients within 2T, so each
 * sample runs orc_diff_grad_f64 on the (4T+1)^2 window around it. */
int orc_diff_lightcone_f64(int64_t NY, int64_t NX, uint64_t seed, uint64_t stream_u, uint64_t stream_k,
                           int T, int64_t nsamp, const int64_t *si, const int64_t *sj, double *uT_out,
                           double *du0_out, double *dk_out) {
    int failed = 0;
    uint64_t ku = orc_stream_key(seed, stream_u), kk = orc_stream_key(seed, stream_k);
    int64_t R = 2 * (int64_t)T;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
    for (int64_t s = 0; s < nsamp; ++s) {
        int64_t r0 = si[s] - R < 0 ? 0 : si[s] - R;
        int64_t r1 = si[s] + R > NY - 1 ? NY - 1 : si[s] + R;
        int64_t c0 = sj[s] - R < 0 ? 0 : sj[s] - R;
        int64_t c1 = sj[s] + R > NX - 1 ? NX - 1 : sj[s] + R;
        int64_t h = r1 - r0 + 1, w = c1 - c0 + 1;
        size_t n = (size_t)(h * w);
        double *u0 = (double *)malloc(n * sizeof(double)), *kap = (double *)malloc(n * sizeof(double));
        double *du = (double *)malloc(n * sizeof(double)), *dk = (double *)malloc(n * sizeof(double));
        double *uT = (double *)malloc(n * sizeof(double));
        if (!u0 || !kap || !du || !dk || !uT) {
            free(u0); free(kap); free(du); free(dk); free(uT);
            failed |= 1;
            continue;
        }
        for (int64_t r = 0; r < h; ++r)
            for (int64_t c = 0; c < w; ++c) {
                uint64_t g = (uint64_t)((r0 + r) * NX + (c0 + c));
                u0[r * w + c] = (double)orc_u01_f32(orc_elem(ku, g));
                kap[r * w + c] = (double)orc_kappa_of(orc_elem(kk, g));
            }
        double J;
        if (orc_diff_grad_f64(h, w, u0, kap, T, &J, du, dk) != 0 ||
            orc_diff_forward_f64(h, w, u0, kap, T, uT) != 0) {
            failed |= 1;
        } else {
            int64_t o = (si[s] - r0) * w + (sj[s] - c0);
            uT_out[s] = uT[o];
            du0_out[s] = du[o];
            dk_out[s] = dk[o];
        }
        free(u0); free(kap); free(du); free(dk); free(uT);
    }
    return failed ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* K-Means (Lloyd's algorithm), as the K-Means benchmark of Sec. 4 runs it:  */
/* n records of 4 f32 features (record i = x[4i .. 4i+3]) and k centres      */
/* (c[4j .. 4j+3]).  The paper computes the centres on the GPU with a        */
/* reduction; one iteration is                                               */
/*  assignment: every record joins its nearest centre by squared Euclidean   */
/*   distance in f32: with d_f = x_f - c_f, dist = fma(d3, d3, fma(d2, d2,   */
/*   fma(d1, d1, d0 * d0))) (each operation rounded once), ties going to     */
/*   the lowest centre index;                                                */
/*  reduction: per centre the fp64 sums of its records' features and their  */
/*   count, s[5j .. 5j+3] and s[5j+4];                                       */
/*  update: centre j becomes f32(sum / count) (fp64 division, then rounded   */
/*   to f32), or keeps its value when no record chose it.                    */
/* ------------------------------------------------------------------------ */
void orc_kmeans_assign(int64_t n, int64_t k, const float *x, const float *c, double *s, int32_t *label) {
    memset(s, 0, (size_t)(5 * k) * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        const float *r = x + 4 * i;
        int64_t best = 0;
        float bd = 0.0f;
        for (int64_t j = 0; j < k; ++j) {
            const float *m = c + 4 * j;
            float d0 = r[0] - m[0], d1 = r[1] - m[1], d2 = r[2] - m[2], d3 = r[3] - m[3];
            float d = fmaf(d3, d3, fmaf(d2, d2, fmaf(d1, d1, d0 * d0)));
            if (j == 0 || d < bd) {
                bd = d;
                best = j;
            }
        }
        for (int f = 0; f < 4; ++f) s[5 * best + f] += (double)r[f];
        s[5 * best + 4] += 1.0;
        if (label) label[i] = (int32_t)best;
    }
}

void orc_kmeans_update(int64_t k, const double *s, const float *c, float *c_new) {
    for (int64_t j = 0; j < k; ++j) {
        double cnt = s[5 * j + 4];
        for (int f = 0; f < 4; ++f) c_new[4 * j + f] = cnt > 0.0 ? (float)(s[5 * j + f] / cnt) : c[4 * j + f];
    }
}
