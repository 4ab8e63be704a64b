/*
 * oracle.c -- plain CPU oracle for the range-mapped kernel path.
 *
 * TEST INFRASTRUCTURE ONLY.  liboracle.so is loaded by the test-suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark, nothing else.  The
 * product library (libsy.so) never links, loads or calls it, and the two share
 * no source, header, table or constant generator.
 *
 * Every routine is the plain definition evaluated in the obvious order.  The file
 * is compiled with -O2 -ffp-contract=off -fno-fast-math, so every float/double
 * operation below is exactly one IEEE-754 round-to-nearest-even operation (no
 * fused multiply-add).  Row loops may run under OpenMP; each output point is
 * computed independently, so the thread count never changes a result.
 *
 * Contents and sources
 *   1. SAXPY  z = alpha*x + y            -- paper §2 Listing 1 (also §3 Listing 2,
 *                                           §4 Listing 3).  FP32 form computes
 *                                           fl(fl(alpha*x) + y), no contraction.
 *   2. Range mappers and row splitting   -- paper §3 (range mapper ties a chunk of
 *                                           the execution range to the data it
 *                                           touches; kernels are split across
 *                                           devices).  one_to_one: chunk [a,b)
 *                                           touches [a,b).  neighbourhood(r): reads
 *                                           [a-r, b+r) clipped to the domain.
 *   3. Central second-difference weights of order 2r (Fornberg, Math. Comp. 51
 *      (1988) 699-706): w_k = 2(-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!), k>=1,
 *      and w_0 = -2 sum_k w_k (so constants are annihilated).
 *   4. Leapfrog wave step in FP64 on an ny x nx grid, star stencil of radius r,
 *      Dirichlet-zero ghost points outside the grid:
 *        L u_ij   = 2 w_0 u_ij + sum_k w_k ((u_{i-k,j}+u_{i+k,j}) + (u_{i,j-k}+u_{i,j+k}))
 *        u^{n+1}  = (2 u^n - u^{n-1}) + c2 * L u^n,   c2 = (c dt/dx)^2
 *      Start with zero initial velocity (second-order Taylor start):
 *        u^{-1}   = u^0 + (c2/2) * L u^0
 *   5. The same step as a precision mirror: storage FP32, BF16 or FP16, values
 *      widened to FP32, the formula above evaluated in FP32 in exactly that
 *      operation order (coefficients rounded once to FP32), the result rounded
 *      once to storage with round-to-nearest-even.
 *   6. Discrete energy (exactly conserved by the recurrence when L is symmetric):
 *        E^{n+1/2} = sum (u^{n+1}-u^n)^2 - c2 * sum u^{n+1} (L u^n)      in FP64.
 *   7. MLP cost model, 3 layers: h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2),
 *      y = W3 h2 + b3; loss = mean over all outputs of (y - t)^2; Adam.  FP64.
 *   8. The leapfrog step of sections 4-6 on an nz x ny x nx grid (a second
 *      workload): the operator is the sum of three one-dimensional second
 *      differences; FP64, precision mirror and energy.
 *   9. Range mappers on 3D boxes (one_to_one from paper §3 Listing 2; the
 *      others are this build's) and the transfers a chunk list implies.
 *
 * The wave workloads, the reduced-precision storage and the cost model are not in
 * the paper; the readings used for them are the ones stated above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_API __attribute__((visibility("default")))

enum { ORACLE_F32 = 0, ORACLE_BF16 = 1, ORACLE_F16 = 2 };

ORACLE_API int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

ORACLE_API void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* 1. SAXPY (paper §2 Listing 1)                                              */
/* ------------------------------------------------------------------------- */

ORACLE_API void oracle_saxpy_f32(int64_t n, float alpha, const float* x, const float* y, float* z) {
    for (int64_t i = 0; i < n; ++i) {
        float ax = alpha * x[i];
        z[i] = ax + y[i];
    }
}

ORACLE_API void oracle_saxpy_f64(int64_t n, double alpha, const double* x, const double* y, double* z) {
    for (int64_t i = 0; i < n; ++i) z[i] = alpha * x[i] + y[i];
}

/* ------------------------------------------------------------------------- */
/* 2. Range mappers and row splitting (paper §3, Listing 2)                   */
/* ------------------------------------------------------------------------- */

/* Even split of [0, ny) into k consecutive chunks; the first ny % k chunks get
 * one extra row.  out holds k (begin, end) pairs. */
ORACLE_API int oracle_split_rows(int64_t ny, int k, int64_t* out) {
    if (ny < 0 || k < 1) return -1;
    int64_t base = ny / k, extra = ny % k, row = 0;
    for (int c = 0; c < k; ++c) {
        int64_t len = base + (c < extra ? 1 : 0);
        out[2 * c] = row;
        out[2 * c + 1] = row + len;
        row += len;
    }
    return 0;
}

/* one_to_one: the chunk touches exactly its own rows. */
ORACLE_API void oracle_rm_one_to_one(int64_t a, int64_t b, int64_t* lo, int64_t* hi) {
    *lo = a;
    *hi = b;
}

/* neighbourhood(r): the chunk reads its rows and r rows on either side,
 * clipped to the domain [0, ny). */
ORACLE_API void oracle_rm_neighbourhood(int64_t a, int64_t b, int r, int64_t ny, int64_t* lo, int64_t* hi) {
    int64_t l = a - r, h = b + r;
    *lo = l < 0 ? 0 : l;
    *hi = h > ny ? ny : h;
}

/* A chunk list is valid when it tiles [0, ny) in order with non-empty chunks. */
ORACLE_API int oracle_chunks_valid(int64_t ny, const int64_t* chunks, int k) {
    if (k < 1) return 0;
    int64_t expect = 0;
    for (int c = 0; c < k; ++c) {
        if (chunks[2 * c] != expect) return 0;
        if (chunks[2 * c + 1] <= chunks[2 * c]) return 0;
        expect = chunks[2 * c + 1];
    }
    return expect == ny;
}

/* ------------------------------------------------------------------------- */
/* 3. Second-difference weights of order 2r                                   */
/* ------------------------------------------------------------------------- */

static double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

ORACLE_API int oracle_d2_weights(int r, double* w) {
    if (r < 1 || r > 4) return -1;
    double sum = 0.0;
    for (int k = 1; k <= r; ++k) {
        double sign = (k % 2 == 1) ? 1.0 : -1.0;
        double num = 2.0 * sign * factorial(r) * factorial(r);
        double den = (double)k * (double)k * factorial(r - k) * factorial(r + k);
        w[k] = num / den;
        sum += w[k];
    }
    w[0] = -2.0 * sum;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 4. Leapfrog wave step, FP64                                                */
/* ------------------------------------------------------------------------- */

static inline double ghost64(const double* u, int64_t ny, int64_t nx, int64_t i, int64_t j) {
    if (i < 0 || i >= ny || j < 0 || j >= nx) return 0.0; /* Dirichlet-zero ghost */
    return u[i * nx + j];
}

static double lap64(const double* u, int64_t ny, int64_t nx, int r, const double* w, int64_t i, int64_t j) {
    double acc = (2.0 * w[0]) * u[i * nx + j];
    for (int k = 1; k <= r; ++k) {
        double vert = ghost64(u, ny, nx, i - k, j) + ghost64(u, ny, nx, i + k, j);
        double horz = ghost64(u, ny, nx, i, j - k) + ghost64(u, ny, nx, i, j + k);
        acc = acc + w[k] * (vert + horz);
    }
    return acc;
}

/* u_next may be the same array as u_prev (each point reads its own u_prev
 * before writing it); it must not be u_cur. */
ORACLE_API int oracle_wave_step_f64(int64_t ny, int64_t nx, int r, double c2, const double* u_prev,
                                    const double* u_cur, double* u_next) {
    double w[5];
    if (oracle_d2_weights(r, w)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; ++i) {
        for (int64_t j = 0; j < nx; ++j) {
            double u = u_cur[i * nx + j];
            u_next[i * nx + j] = (2.0 * u - u_prev[i * nx + j]) + c2 * lap64(u_cur, ny, nx, r, w, i, j);
        }
    }
    return 0;
}

/* Taylor start for zero initial velocity: u^{-1} = u^0 + (c2/2) L u^0. */
ORACLE_API int oracle_wave_start_f64(int64_t ny, int64_t nx, int r, double c2, const double* u0, double* um1) {
    double w[5];
    if (oracle_d2_weights(r, w)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; ++i)
        for (int64_t j = 0; j < nx; ++j)
            um1[i * nx + j] = u0[i * nx + j] + (0.5 * c2) * lap64(u0, ny, nx, r, w, i, j);
    return 0;
}

/* Start, then `steps` leapfrog steps.  On return prev = u^{steps-1} and
 * cur = u^{steps} (steps = 0 gives prev = u^{-1}, cur = u^0). */
ORACLE_API int oracle_wave_run_f64(int64_t ny, int64_t nx, int r, double c2, int64_t steps, const double* u0,
                                   double* prev, double* cur) {
    int64_t n = ny * nx;
    if (oracle_wave_start_f64(ny, nx, r, c2, u0, prev)) return -1;
    memcpy(cur, u0, (size_t)n * sizeof(double));
    for (int64_t s = 0; s < steps; ++s) {
        /* u^{s+1} overwrites u^{s-1}; then swap roles by swapping contents. */
        if (oracle_wave_step_f64(ny, nx, r, c2, prev, cur, prev)) return -1;
        for (int64_t p = 0; p < n; ++p) {
            double t = prev[p];
            prev[p] = cur[p];
            cur[p] = t;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 5. Precision mirror: FP32 compute, FP32/BF16/FP16 storage                  */
/* ------------------------------------------------------------------------- */

static float f32_from_bits(uint32_t b) {
    float f;
    memcpy(&f, &b, 4);
    return f;
}

static uint32_t bits_from_f32(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

/* bfloat16 = the upper 16 bits of a binary32; rounding adds half an ulp of the
 * kept part (0x7fff) plus the kept part's lowest bit, which breaks ties to even. */
ORACLE_API uint16_t oracle_f32_to_bf16(float f) {
    uint32_t b = bits_from_f32(f);
    if ((b & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((b >> 16) | 0x0040u); /* quiet NaN */
    uint32_t keep_lsb = (b >> 16) & 1u;
    b += 0x7fffu + keep_lsb;
    return (uint16_t)(b >> 16);
}

ORACLE_API float oracle_bf16_to_f32(uint16_t h) { return f32_from_bits((uint32_t)h << 16); }

/* binary16 from binary32 with round-to-nearest-even, written from the format's
 * definition: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits; normal
 * values 2^(e-15) * 1.f for e in 1..30, subnormals 2^-14 * 0.f.  The value is
 * rounded in double arithmetic, which is exact here: |f| * 2^24 is an integer
 * multiple of the spacing, and nearbyint() rounds half to even. */
ORACLE_API uint16_t oracle_f32_to_f16(float f) {
    uint32_t b = bits_from_f32(f);
    uint16_t sign = (uint16_t)((b >> 16) & 0x8000u);
    if ((b & 0x7fffffffu) > 0x7f800000u) return (uint16_t)(sign | 0x7e00u); /* quiet NaN */
    double a = fabs((double)f);
    if (a == 0.0) return sign;
    if (isinf(a)) return (uint16_t)(sign | 0x7c00u);
    /* exponent of the binade holding a, clamped to the subnormal binade */
    int e;
    frexp(a, &e); /* a = m * 2^e, m in [0.5, 1): binade exponent is e-1 */
    int binade = e - 1;
    if (binade < -14) binade = -14;
    double quantum = ldexp(1.0, binade - 10); /* spacing of binary16 values there */
    double n = nearbyint(a / quantum);         /* round half to even */
    double v = n * quantum;
    if (v > 65504.0) return (uint16_t)(sign | 0x7c00u); /* past the largest finite value: infinity */
    if (v < ldexp(1.0, -14)) {
        /* subnormal (or rounds up to the smallest normal when n == 1024) */
        return (uint16_t)(sign | (uint16_t)(v / ldexp(1.0, -24)));
    }
    frexp(v, &e);
    int E = (e - 1) + 15;
    double frac = v / ldexp(1.0, e - 1) - 1.0; /* in [0, 1) */
    uint16_t mant = (uint16_t)(frac * 1024.0);
    return (uint16_t)(sign | (uint16_t)(E << 10) | mant);
}

ORACLE_API float oracle_f16_to_f32(uint16_t h) {
    int sign = (h >> 15) & 1;
    int E = (h >> 10) & 0x1f;
    int mant = h & 0x3ff;
    double v;
    if (E == 0)
        v = ldexp((double)mant, -24);
    else if (E == 31)
        v = mant ? NAN : INFINITY;
    else
        v = ldexp(1.0 + mant / 1024.0, E - 15);
    return (float)(sign ? -v : v);
}

static inline float load_storage(int dtype, const void* p, int64_t idx) {
    if (dtype == ORACLE_F32) return ((const float*)p)[idx];
    uint16_t h = ((const uint16_t*)p)[idx];
    return dtype == ORACLE_BF16 ? oracle_bf16_to_f32(h) : oracle_f16_to_f32(h);
}

static inline void store_storage(int dtype, void* p, int64_t idx, float v) {
    if (dtype == ORACLE_F32)
        ((float*)p)[idx] = v;
    else if (dtype == ORACLE_BF16)
        ((uint16_t*)p)[idx] = oracle_f32_to_bf16(v);
    else
        ((uint16_t*)p)[idx] = oracle_f32_to_f16(v);
}

static inline float ghost_m(int dtype, const void* u, int64_t ny, int64_t nx, int64_t i, int64_t j) {
    if (i < 0 || i >= ny || j < 0 || j >= nx) return 0.0f;
    return load_storage(dtype, u, i * nx + j);
}

static float lap_m(int dtype, const void* u, int64_t ny, int64_t nx, int r, const float* wf, float c0x2, int64_t i,
                   int64_t j) {
    float acc = c0x2 * load_storage(dtype, u, i * nx + j);
    for (int k = 1; k <= r; ++k) {
        float vert = ghost_m(dtype, u, ny, nx, i - k, j) + ghost_m(dtype, u, ny, nx, i + k, j);
        float horz = ghost_m(dtype, u, ny, nx, i, j - k) + ghost_m(dtype, u, ny, nx, i, j + k);
        float pair = vert + horz;
        float term = wf[k] * pair;
        acc = acc + term;
    }
    return acc;
}

static int mirror_weights(int r, float* wf, float* c0x2) {
    double w[5];
    if (oracle_d2_weights(r, w)) return -1;
    for (int k = 1; k <= r; ++k) wf[k] = (float)w[k];
    *c0x2 = (float)(2.0 * w[0]);
    return 0;
}

ORACLE_API int oracle_wave_step_mirror(int dtype, int64_t ny, int64_t nx, int r, float c2, const void* u_prev,
                                       const void* u_cur, void* u_next) {
    float wf[5], c0x2;
    if (mirror_weights(r, wf, &c0x2)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; ++i) {
        for (int64_t j = 0; j < nx; ++j) {
            float u = load_storage(dtype, u_cur, i * nx + j);
            float up = load_storage(dtype, u_prev, i * nx + j);
            float lap = lap_m(dtype, u_cur, ny, nx, r, wf, c0x2, i, j);
            float two_u = 2.0f * u;
            float inertia = two_u - up;
            float force = c2 * lap;
            store_storage(dtype, u_next, i * nx + j, inertia + force);
        }
    }
    return 0;
}

ORACLE_API int oracle_wave_start_mirror(int dtype, int64_t ny, int64_t nx, int r, float c2, const void* u0,
                                        void* um1) {
    float wf[5], c0x2;
    if (mirror_weights(r, wf, &c0x2)) return -1;
    float half_c2 = 0.5f * c2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; ++i) {
        for (int64_t j = 0; j < nx; ++j) {
            float u = load_storage(dtype, u0, i * nx + j);
            float lap = lap_m(dtype, u0, ny, nx, r, wf, c0x2, i, j);
            float force = half_c2 * lap;
            store_storage(dtype, um1, i * nx + j, u + force);
        }
    }
    return 0;
}

ORACLE_API int oracle_wave_run_mirror(int dtype, int64_t ny, int64_t nx, int r, float c2, int64_t steps,
                                      const void* u0, void* prev, void* cur) {
    size_t esz = dtype == ORACLE_F32 ? 4 : 2;
    size_t bytes = (size_t)(ny * nx) * esz;
    if (oracle_wave_start_mirror(dtype, ny, nx, r, c2, u0, prev)) return -1;
    memcpy(cur, u0, bytes);
    void* tmp = malloc(bytes ? bytes : 1);
    if (!tmp) return -2;
    for (int64_t s = 0; s < steps; ++s) {
        if (oracle_wave_step_mirror(dtype, ny, nx, r, c2, prev, cur, prev)) {
            free(tmp);
            return -1;
        }
        memcpy(tmp, prev, bytes);
        memcpy(prev, cur, bytes);
        memcpy(cur, tmp, bytes);
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 6. Discrete energy, FP64                                                   */
/* ------------------------------------------------------------------------- */

/* E = kin - c2 * pot with kin = sum (u_new - u_old)^2 and pot = sum u_new (L u_old),
 * both summed sequentially in row-major order.  abs_sum receives
 * sum |(u_new-u_old)^2| + c2 * sum |u_new (L u_old)| (the size of the terms,
 * used to bound rounding differences of other summation orders). */
ORACLE_API double oracle_wave_energy_f64(int64_t ny, int64_t nx, int r, double c2, const double* u_new,
                                         const double* u_old, double* kin_out, double* pot_out, double* abs_sum) {
    double w[5];
    if (oracle_d2_weights(r, w)) return NAN;
    double kin = 0.0, pot = 0.0, mag = 0.0;
    for (int64_t i = 0; i < ny; ++i) {
        for (int64_t j = 0; j < nx; ++j) {
            double d = u_new[i * nx + j] - u_old[i * nx + j];
            double p = u_new[i * nx + j] * lap64(u_old, ny, nx, r, w, i, j);
            kin += d * d;
            pot += p;
            mag += d * d + c2 * fabs(p);
        }
    }
    if (kin_out) *kin_out = kin;
    if (pot_out) *pot_out = pot;
    if (abs_sum) *abs_sum = mag;
    return kin - c2 * pot;
}

/* ------------------------------------------------------------------------- */
/* 7. MLP cost model, FP64                                                    */
/* ------------------------------------------------------------------------- */
/* Parameter vector layout (row-major, out x in):
 *   W1[H][F], b1[H], W2[H][H], b2[H], W3[O][H], b3[O]                         */

static double silu(double z) { return z / (1.0 + exp(-z)); }

static double silu_grad(double z) {
    double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

ORACLE_API int64_t oracle_mlp_param_count(int F, int H, int O) {
    return (int64_t)H * F + H + (int64_t)H * H + H + (int64_t)O * H + O;
}

typedef struct {
    const double *W1, *b1, *W2, *b2, *W3, *b3;
} mlp_view;

static mlp_view mlp_split(const double* p, int F, int H, int O) {
    mlp_view v;
    v.W1 = p;
    v.b1 = v.W1 + (int64_t)H * F;
    v.W2 = v.b1 + H;
    v.b2 = v.W2 + (int64_t)H * H;
    v.W3 = v.b2 + H;
    v.b3 = v.W3 + (int64_t)O * H;
    return v;
}

/* Forward for one sample; z1,h1,z2,h2 (H each) and y (O) are outputs. */
static void mlp_forward_one(const mlp_view* m, int F, int H, int O, const double* x, double* z1, double* h1,
                            double* z2, double* h2, double* y) {
    for (int j = 0; j < H; ++j) {
        double s = m->b1[j];
        for (int i = 0; i < F; ++i) s += m->W1[(int64_t)j * F + i] * x[i];
        z1[j] = s;
        h1[j] = silu(s);
    }
    for (int j = 0; j < H; ++j) {
        double s = m->b2[j];
        for (int i = 0; i < H; ++i) s += m->W2[(int64_t)j * H + i] * h1[i];
        z2[j] = s;
        h2[j] = silu(s);
    }
    for (int o = 0; o < O; ++o) {
        double s = m->b3[o];
        for (int i = 0; i < H; ++i) s += m->W3[(int64_t)o * H + i] * h2[i];
        y[o] = s;
    }
}

ORACLE_API int oracle_mlp_forward(int64_t B, int F, int H, int O, const double* X, const double* params,
                                  double* Y) {
    if (H > 4096) return -1;
    mlp_view m = mlp_split(params, F, H, O);
    double* work = (double*)malloc(sizeof(double) * (size_t)(4 * H + 1));
    if (!work) return -2;
    for (int64_t b = 0; b < B; ++b)
        mlp_forward_one(&m, F, H, O, X + b * F, work, work + H, work + 2 * H, work + 3 * H, Y + b * O);
    free(work);
    return 0;
}

/* loss = (1 / (B*O)) * sum_b sum_o (y_bo - t_bo)^2; grad has the layout of
 * params and receives d loss / d params (overwritten).  Returns the loss. */
ORACLE_API double oracle_mlp_loss_grad(int64_t B, int F, int H, int O, const double* X, const double* T,
                                       const double* params, double* grad) {
    mlp_view m = mlp_split(params, F, H, O);
    int64_t P = oracle_mlp_param_count(F, H, O);
    memset(grad, 0, sizeof(double) * (size_t)P);
    double *gW1 = grad, *gb1 = gW1 + (int64_t)H * F, *gW2 = gb1 + H, *gb2 = gW2 + (int64_t)H * H;
    double *gW3 = gb2 + H, *gb3 = gW3 + (int64_t)O * H;
    double* work = (double*)malloc(sizeof(double) * (size_t)(7 * H + 2 * O + 1));
    if (!work) return NAN;
    double *z1 = work, *h1 = z1 + H, *z2 = h1 + H, *h2 = z2 + H, *y = h2 + H;
    double *dy = y + O, *dh2 = dy + O, *dz1 = dh2 + H, *dz2 = dz1 + H;
    double loss = 0.0, scale = 1.0 / ((double)B * (double)O);
    for (int64_t b = 0; b < B; ++b) {
        const double* x = X + b * F;
        mlp_forward_one(&m, F, H, O, x, z1, h1, z2, h2, y);
        for (int o = 0; o < O; ++o) {
            double e = y[o] - T[b * O + o];
            loss += e * e;
            dy[o] = 2.0 * e * scale;
        }
        /* layer 3: y = W3 h2 + b3 */
        for (int o = 0; o < O; ++o) {
            gb3[o] += dy[o];
            for (int i = 0; i < H; ++i) gW3[(int64_t)o * H + i] += dy[o] * h2[i];
        }
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int o = 0; o < O; ++o) s += m.W3[(int64_t)o * H + i] * dy[o];
            dh2[i] = s;
        }
        /* layer 2: h2 = silu(z2), z2 = W2 h1 + b2 */
        for (int j = 0; j < H; ++j) dz2[j] = dh2[j] * silu_grad(z2[j]);
        for (int j = 0; j < H; ++j) {
            gb2[j] += dz2[j];
            for (int i = 0; i < H; ++i) gW2[(int64_t)j * H + i] += dz2[j] * h1[i];
        }
        /* layer 1: h1 = silu(z1), z1 = W1 x + b1 */
        for (int i = 0; i < H; ++i) {
            double s = 0.0;
            for (int j = 0; j < H; ++j) s += m.W2[(int64_t)j * H + i] * dz2[j];
            dz1[i] = s * silu_grad(z1[i]);
        }
        for (int j = 0; j < H; ++j) {
            gb1[j] += dz1[j];
            for (int i = 0; i < F; ++i) gW1[(int64_t)j * F + i] += dz1[j] * x[i];
        }
    }
    free(work);
    return loss * scale;
}

/* One Adam step (Kingma & Ba 2015, Algorithm 1) on n parameters; t is the
 * 1-based step number after this update. */
ORACLE_API void oracle_adam_step(int64_t n, double* params, const double* grad, double* m, double* v, int64_t t,
                                 double lr, double beta1, double beta2, double eps) {
    double bc1 = 1.0 - pow(beta1, (double)t);
    double bc2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mhat = m[i] / bc1;
        double vhat = v[i] / bc2;
        params[i] -= lr * mhat / (sqrt(vhat) + eps);
    }
}

/* ------------------------------------------------------------------------- */
/* 8. Leapfrog wave step in 3D (second workload), FP64 and precision mirror   */
/* ------------------------------------------------------------------------- */
/* Grid nz x ny x nx, point (k, i, j) at (k*ny + i)*nx + j.  The operator is the
 * sum of the three one-dimensional second differences of section 3, each with its
 * own w_0 term, Dirichlet-zero ghosts in every direction:
 *   L u = 3 w_0 u + sum_m w_m ( ((u_{k,i-m,j}+u_{k,i+m,j}) + (u_{k,i,j-m}+u_{k,i,j+m}))
 *                               + (u_{k-m,i,j}+u_{k+m,i,j}) )
 * The recurrence and the start are those of section 4; the mirror evaluates the
 * bracketing above in FP32, 3 w_0 rounded once to FP32. */

static inline double ghost3(const double* u, int64_t nz, int64_t ny, int64_t nx, int64_t k, int64_t i, int64_t j) {
    if (k < 0 || k >= nz || i < 0 || i >= ny || j < 0 || j >= nx) return 0.0;
    return u[(k * ny + i) * nx + j];
}

static double lap3_64(const double* u, int64_t nz, int64_t ny, int64_t nx, int r, const double* w, int64_t k,
                      int64_t i, int64_t j) {
    double acc = (3.0 * w[0]) * u[(k * ny + i) * nx + j];
    for (int m = 1; m <= r; ++m) {
        double vert = ghost3(u, nz, ny, nx, k, i - m, j) + ghost3(u, nz, ny, nx, k, i + m, j);
        double horz = ghost3(u, nz, ny, nx, k, i, j - m) + ghost3(u, nz, ny, nx, k, i, j + m);
        double depth = ghost3(u, nz, ny, nx, k - m, i, j) + ghost3(u, nz, ny, nx, k + m, i, j);
        acc = acc + w[m] * ((vert + horz) + depth);
    }
    return acc;
}

/* u_next may be u_prev; it must not be u_cur. */
ORACLE_API int oracle_wave3d_step_f64(int64_t nz, int64_t ny, int64_t nx, int r, double c2, const double* u_prev,
                                      const double* u_cur, double* u_next) {
    double w[5];
    if (oracle_d2_weights(r, w)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                int64_t p = (k * ny + i) * nx + j;
                double u = u_cur[p];
                u_next[p] = (2.0 * u - u_prev[p]) + c2 * lap3_64(u_cur, nz, ny, nx, r, w, k, i, j);
            }
    return 0;
}

ORACLE_API int oracle_wave3d_start_f64(int64_t nz, int64_t ny, int64_t nx, int r, double c2, const double* u0,
                                       double* um1) {
    double w[5];
    if (oracle_d2_weights(r, w)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                int64_t p = (k * ny + i) * nx + j;
                um1[p] = u0[p] + (0.5 * c2) * lap3_64(u0, nz, ny, nx, r, w, k, i, j);
            }
    return 0;
}

/* Start, then `steps` steps: prev = u^{steps-1}, cur = u^{steps}. */
ORACLE_API int oracle_wave3d_run_f64(int64_t nz, int64_t ny, int64_t nx, int r, double c2, int64_t steps,
                                     const double* u0, double* prev, double* cur) {
    int64_t n = nz * ny * nx;
    if (oracle_wave3d_start_f64(nz, ny, nx, r, c2, u0, prev)) return -1;
    memcpy(cur, u0, (size_t)n * sizeof(double));
    for (int64_t s = 0; s < steps; ++s) {
        if (oracle_wave3d_step_f64(nz, ny, nx, r, c2, prev, cur, prev)) return -1;
        for (int64_t p = 0; p < n; ++p) {
            double t = prev[p];
            prev[p] = cur[p];
            cur[p] = t;
        }
    }
    return 0;
}

static inline float ghost3_m(int dtype, const void* u, int64_t nz, int64_t ny, int64_t nx, int64_t k, int64_t i,
                             int64_t j) {
    if (k < 0 || k >= nz || i < 0 || i >= ny || j < 0 || j >= nx) return 0.0f;
    return load_storage(dtype, u, (k * ny + i) * nx + j);
}

static float lap3_m(int dtype, const void* u, int64_t nz, int64_t ny, int64_t nx, int r, const float* wf, float c0x3,
                    int64_t k, int64_t i, int64_t j) {
    float acc = c0x3 * load_storage(dtype, u, (k * ny + i) * nx + j);
    for (int m = 1; m <= r; ++m) {
        float vert = ghost3_m(dtype, u, nz, ny, nx, k, i - m, j) + ghost3_m(dtype, u, nz, ny, nx, k, i + m, j);
        float horz = ghost3_m(dtype, u, nz, ny, nx, k, i, j - m) + ghost3_m(dtype, u, nz, ny, nx, k, i, j + m);
        float depth = ghost3_m(dtype, u, nz, ny, nx, k - m, i, j) + ghost3_m(dtype, u, nz, ny, nx, k + m, i, j);
        float plane = vert + horz;
        float pair = plane + depth;
        float term = wf[m] * pair;
        acc = acc + term;
    }
    return acc;
}

static int mirror_weights3(int r, float* wf, float* c0x3) {
    double w[5];
    if (oracle_d2_weights(r, w)) return -1;
    for (int m = 1; m <= r; ++m) wf[m] = (float)w[m];
    *c0x3 = (float)(3.0 * w[0]);
    return 0;
}

ORACLE_API int oracle_wave3d_step_mirror(int dtype, int64_t nz, int64_t ny, int64_t nx, int r, float c2,
                                         const void* u_prev, const void* u_cur, void* u_next) {
    float wf[5], c0x3;
    if (mirror_weights3(r, wf, &c0x3)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                int64_t p = (k * ny + i) * nx + j;
                float u = load_storage(dtype, u_cur, p);
                float up = load_storage(dtype, u_prev, p);
                float lap = lap3_m(dtype, u_cur, nz, ny, nx, r, wf, c0x3, k, i, j);
                float two_u = 2.0f * u;
                float inertia = two_u - up;
                float force = c2 * lap;
                store_storage(dtype, u_next, p, inertia + force);
            }
    return 0;
}

ORACLE_API int oracle_wave3d_start_mirror(int dtype, int64_t nz, int64_t ny, int64_t nx, int r, float c2,
                                          const void* u0, void* um1) {
    float wf[5], c0x3;
    if (mirror_weights3(r, wf, &c0x3)) return -1;
    float half_c2 = 0.5f * c2;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                int64_t p = (k * ny + i) * nx + j;
                float u = load_storage(dtype, u0, p);
                float lap = lap3_m(dtype, u0, nz, ny, nx, r, wf, c0x3, k, i, j);
                float force = half_c2 * lap;
                store_storage(dtype, um1, p, u + force);
            }
    return 0;
}

ORACLE_API int oracle_wave3d_run_mirror(int dtype, int64_t nz, int64_t ny, int64_t nx, int r, float c2,
                                        int64_t steps, const void* u0, void* prev, void* cur) {
    size_t esz = dtype == ORACLE_F32 ? 4 : 2;
    size_t bytes = (size_t)(nz * ny * nx) * esz;
    if (oracle_wave3d_start_mirror(dtype, nz, ny, nx, r, c2, u0, prev)) return -1;
    memcpy(cur, u0, bytes);
    void* tmp = malloc(bytes ? bytes : 1);
    if (!tmp) return -2;
    for (int64_t s = 0; s < steps; ++s) {
        if (oracle_wave3d_step_mirror(dtype, nz, ny, nx, r, c2, prev, cur, prev)) {
            free(tmp);
            return -1;
        }
        memcpy(tmp, prev, bytes);
        memcpy(prev, cur, bytes);
        memcpy(cur, tmp, bytes);
    }
    free(tmp);
    return 0;
}

/* Discrete energy of section 6 with the 3D operator. */
ORACLE_API double oracle_wave3d_energy_f64(int64_t nz, int64_t ny, int64_t nx, int r, double c2, const double* u_new,
                                           const double* u_old, double* kin_out, double* pot_out) {
    double w[5];
    if (oracle_d2_weights(r, w)) return NAN;
    double kin = 0.0, pot = 0.0;
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t i = 0; i < ny; ++i)
            for (int64_t j = 0; j < nx; ++j) {
                int64_t p = (k * ny + i) * nx + j;
                double d = u_new[p] - u_old[p];
                kin += d * d;
                pot += u_new[p] * lap3_64(u_old, nz, ny, nx, r, w, k, i, j);
            }
    if (kin_out) *kin_out = kin;
    if (pot_out) *pot_out = pot;
    return kin - c2 * pot;
}

/* ------------------------------------------------------------------------- */
/* 9. Range mappers on boxes (paper §3: a range mapper ties the chunk of the  */
/*    execution range a device runs to the part of a buffer it accesses)      */
/* ------------------------------------------------------------------------- */
/* A box is [lo_d, hi_d) in each of 3 dimensions, dimension 0 the slowest.  The
 * paper names one_to_one; neighbourhood, slice, all and fixed are this build's
 * other mappers:
 *   one_to_one        chunk -> chunk
 *   neighbourhood(r)  chunk grown by r_d on both sides of dimension d
 *   slice(d)          chunk with dimension d widened to the whole buffer
 *   all               the whole buffer
 *   fixed(B)          the box B
 * every result clipped to the buffer [0, extent_d).  An empty box has lo >= hi
 * in some dimension. */
enum { ORACLE_RM_ONE_TO_ONE = 0, ORACLE_RM_NEIGHBOURHOOD = 1, ORACLE_RM_SLICE = 2, ORACLE_RM_ALL = 3,
       ORACLE_RM_FIXED = 4 };

/* box: lo[3], hi[3] as 6 int64 (lo0, lo1, lo2, hi0, hi1, hi2). */
ORACLE_API int oracle_rm_box(int kind, const int64_t* radius, int dim, const int64_t* fixed, const int64_t* chunk,
                             const int64_t* extent, int64_t* out) {
    for (int d = 0; d < 3; ++d) {
        int64_t lo = chunk[d], hi = chunk[3 + d];
        switch (kind) {
            case ORACLE_RM_ONE_TO_ONE: break;
            case ORACLE_RM_NEIGHBOURHOOD:
                lo -= radius[d];
                hi += radius[d];
                break;
            case ORACLE_RM_SLICE:
                if (d == dim) {
                    lo = 0;
                    hi = extent[d];
                }
                break;
            case ORACLE_RM_ALL:
                lo = 0;
                hi = extent[d];
                break;
            case ORACLE_RM_FIXED:
                lo = fixed[d];
                hi = fixed[3 + d];
                break;
            default: return -1;
        }
        out[d] = lo < 0 ? 0 : lo;
        out[3 + d] = hi > extent[d] ? extent[d] : hi;
    }
    return 0;
}

/* Transfers a chunk list needs before a kernel with this mapper runs, when
 * chunk c owns (holds the current values of) exactly its own box: for every
 * ordered pair (src, dst), src != dst, the box rm(chunk_dst) intersected with
 * chunk_src, if non-empty.  Written in dst-major, src-minor order as
 * (src, dst, box[6]) records of 8 int64; returns how many, or -1 if more than
 * max_out. */
ORACLE_API int oracle_rm_box_transfers(int kind, const int64_t* radius, int dim, const int64_t* fixed,
                                       const int64_t* chunks, int n, const int64_t* extent, int64_t* out,
                                       int max_out) {
    int count = 0;
    for (int dst = 0; dst < n; ++dst) {
        int64_t need[6];
        if (oracle_rm_box(kind, radius, dim, fixed, chunks + 6 * dst, extent, need)) return -1;
        for (int src = 0; src < n; ++src) {
            if (src == dst) continue;
            const int64_t* own = chunks + 6 * src;
            int64_t box[6];
            int empty = 0;
            for (int d = 0; d < 3; ++d) {
                box[d] = need[d] > own[d] ? need[d] : own[d];
                box[3 + d] = need[3 + d] < own[3 + d] ? need[3 + d] : own[3 + d];
                if (box[d] >= box[3 + d]) empty = 1;
            }
            if (empty) continue;
            if (count >= max_out) return -1;
            int64_t* rec = out + 8 * count;
            rec[0] = src;
            rec[1] = dst;
            for (int q = 0; q < 6; ++q) rec[2 + q] = box[q];
            ++count;
        }
    }
    return count;
}
