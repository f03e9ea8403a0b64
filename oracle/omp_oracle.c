/*
 * CPU oracle for the data-parallel hot path of an OpenMP GPU device runtime
 * ("Experience Report: Writing A Portable GPU Runtime with OpenMP 5.1",
 * arXiv 2106.03219).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or constant with the CUDA library.
 *
 * The paper names the runtime routines this oracle models but does not
 * specify their semantics:
 *   - splitting a worksharing loop's iterations among threads (Sec. 1,
 *     Sec. 2),
 *   - __kmpc_alloc_shared(uint64_t bytes) (Sec. 2.1, Listing 1),
 *   - team = thread block, team-shared variables (Sec. 3.1, "Global Shared
 *     Variables"),
 *   - the five atomics add/inc/max/exchange/cas (Sec. 3.1, Listing 3 and the
 *     inc definition that follows it),
 *   - synchronisation and thread hierarchy (Sec. 3.2).
 * The loop semantics below are the OpenMP loop-schedule rules (OpenMP 5.1,
 * cited in Sec. 3.1) with every implementation-defined point fixed to one
 * stated reading.  Every function names the reading it follows.
 *
 * Floating point: built with -ffp-contract=off so that no multiply-add is
 * fused unless fma()/fmaf() is called explicitly.
 *
 * Parity status: every function here is pinned by the tests under
 * tests/test_oracle_*.py (brute force, closed forms, math.fsum, exact
 * rational arithmetic, finite differences).  None is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* index types of the loop variable                                    */
/* ------------------------------------------------------------------ */
enum { ORC_I32 = 0, ORC_U32 = 1, ORC_I64 = 2, ORC_U64 = 3 };
enum { ORC_OK = 0, ORC_EINVAL = 1 };

static int orc_is_signed(int type) { return type == ORC_I32 || type == ORC_I64; }

/* A bound given as a 64-bit pattern, brought to the 64-bit working value:
 * 32-bit signed types sign-extend, 32-bit unsigned zero-extend. */
static int64_t orc_widen(int64_t v, int type)
{
    if (type == ORC_I32) return (int64_t)(int32_t)v;
    if (type == ORC_U32) return (int64_t)(uint32_t)v;
    return v;
}

/* 64-bit two's-complement helpers: exact modulo 2^64, never undefined. */
static int64_t orc_add(int64_t a, int64_t b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
static int64_t orc_mul(uint64_t a, int64_t b) { return (int64_t)(a * (uint64_t)b); }

/*
 * C0: trip count of  for (v = lb; incr > 0 ? v <= ub : v >= ub; v += incr).
 * Bounds compare in the loop variable's own signedness; the distance is taken
 * in unsigned 64-bit arithmetic so it cannot overflow.  incr == 0, a bound
 * outside the type, or 2^64 iterations are rejected.
 */
int orc_trip_count(int64_t lb, int64_t ub, int64_t incr, int type, uint64_t *n_out)
{
    if (incr == 0 || type < ORC_I32 || type > ORC_U64) return ORC_EINVAL;
    if (type == ORC_I32 && (lb != (int64_t)(int32_t)lb || ub != (int64_t)(int32_t)ub))
        return ORC_EINVAL;
    if (type == ORC_U32 && (lb != (int64_t)(uint32_t)lb || ub != (int64_t)(uint32_t)ub))
        return ORC_EINVAL;
    if ((type == ORC_I32 || type == ORC_U32) && (incr > INT32_MAX || incr < -INT32_MAX))
        return ORC_EINVAL;
    if (incr == INT64_MIN) return ORC_EINVAL;

    int empty;
    if (orc_is_signed(type))
        empty = incr > 0 ? (ub < lb) : (ub > lb);
    else
        empty = incr > 0 ? ((uint64_t)ub < (uint64_t)lb) : ((uint64_t)ub > (uint64_t)lb);
    if (empty) { *n_out = 0; return ORC_OK; }

    uint64_t dist = incr > 0 ? (uint64_t)ub - (uint64_t)lb : (uint64_t)lb - (uint64_t)ub;
    uint64_t step = incr > 0 ? (uint64_t)incr : (uint64_t)0 - (uint64_t)incr;
    uint64_t q = dist / step;
    if (q == UINT64_MAX) return ORC_EINVAL;
    *n_out = q + 1;
    return ORC_OK;
}

/*
 * C1 (static, no chunk): the n logical iterations are cut into P contiguous
 * pieces in entity order, the first n % P pieces one longer.  Entity k starts
 * at logical index k*q + min(k, r) and owns q + (k < r) iterations.
 */
void orc_static_nochunk(uint64_t n, uint64_t P, uint64_t k, uint64_t *start, uint64_t *count)
{
    uint64_t q = n / P, r = n % P;
    *count = q + (k < r ? 1 : 0);
    *start = k * q + (k < r ? k : r);
}

/*
 * Level-agnostic static worksharing over a block of logical iterations
 * [bs, bs + bn) of a loop with user bounds (lb, incr), for entity k of P,
 * chunk c (0 = no chunk).  Produces the __kmpc_for_static_init-style tuple in
 * user index space:
 *   LB, UB  first (or only) piece, inclusive;
 *   stride  distance between the entity's consecutive pieces
 *           (bn*incr without chunk, P*c*incr with chunk);
 *   last    the entity owns the block's final iteration.
 * An entity with no iterations gets LB = lb + (bs+bn)*incr, UB = LB - incr.
 * All arithmetic is 64-bit two's complement on the widened bounds.
 */
static void orc_static_block(int64_t lb, int64_t incr, uint64_t bs, uint64_t bn,
                             uint64_t P, uint64_t k, uint64_t c,
                             int64_t *LB, int64_t *UB, int64_t *stride, int *last)
{
    uint64_t s, cnt;
    if (c == 0) {
        orc_static_nochunk(bn, P, k, &s, &cnt);
        *stride = orc_mul(bn, incr);
        *last = (cnt > 0 && s + cnt == bn);
    } else {
        /* C2: chunk j = [j*c, min((j+1)*c, bn)), owner j mod P */
        uint64_t nch = bn == 0 ? 0 : (bn - 1) / c + 1;
        if (k < nch) {
            s = k * c;
            cnt = (bn - s > c) ? c : bn - s;
        } else {
            s = bn;
            cnt = 0;
        }
        *stride = orc_mul(P * c, incr);
        *last = (nch > 0 && k == (nch - 1) % P);
    }
    if (cnt == 0) s = bn;
    *LB = orc_add(lb, orc_mul(bs + s, incr));
    *UB = cnt > 0 ? orc_add(*LB, orc_mul(cnt - 1, incr)) : orc_add(*LB, -incr);
}

/* Single-level static worksharing (C1 / C2) over the whole loop. */
int orc_for_static_init(int64_t lb, int64_t ub, int64_t incr, int type,
                        uint64_t P, uint64_t k, uint64_t chunk,
                        int64_t *LB, int64_t *UB, int64_t *stride, int *last)
{
    uint64_t n;
    int rc = orc_trip_count(lb, ub, incr, type, &n);
    if (rc) return rc;
    if (P == 0 || k >= P) return ORC_EINVAL;
    orc_static_block(orc_widen(lb, type), incr, 0, n, P, k, chunk, LB, UB, stride, last);
    return ORC_OK;
}

/*
 * C3: composite "teams distribute parallel for".  Level 1 cuts the loop among
 * G teams with C1; level 2 cuts team g's block among T threads with C1 (chunk
 * 0) or C2 (chunk c), chunk numbering restarting at the block start.
 * table: G*T rows of 8 int64: team LB, UB, stride, last, thread LB, UB,
 * stride, last (row g*T + t).
 */
int orc_composite_table(int64_t lb, int64_t ub, int64_t incr, int type,
                        uint64_t G, uint64_t T, uint64_t chunk, int64_t *table)
{
    uint64_t n;
    int rc = orc_trip_count(lb, ub, incr, type, &n);
    if (rc) return rc;
    if (G == 0 || T == 0) return ORC_EINVAL;
    int64_t wlb = orc_widen(lb, type);
    for (uint64_t g = 0; g < G; g++) {
        uint64_t bs, bn;
        int64_t tLB, tUB, tst;
        int tlast;
        orc_static_nochunk(n, G, g, &bs, &bn);
        orc_static_block(wlb, incr, 0, n, G, g, 0, &tLB, &tUB, &tst, &tlast);
        for (uint64_t t = 0; t < T; t++) {
            int64_t LB, UB, st;
            int last;
            orc_static_block(wlb, incr, bs, bn, T, t, chunk, &LB, &UB, &st, &last);
            int64_t *row = table + 8 * (g * T + t);
            row[0] = tLB; row[1] = tUB; row[2] = tst; row[3] = tlast;
            row[4] = LB;  row[5] = UB;  row[6] = st;  row[7] = last;
        }
    }
    return ORC_OK;
}

/*
 * C3 owner map: owner[i] = g*T + t for every logical iteration i in [0, n).
 * Iterations are enumerated one by one from each thread's pieces.
 */
int orc_owner_map(uint64_t n, uint64_t G, uint64_t T, uint64_t chunk, int32_t *owner)
{
    if (G == 0 || T == 0) return ORC_EINVAL;
    for (uint64_t g = 0; g < G; g++) {
        uint64_t bs, bn;
        orc_static_nochunk(n, G, g, &bs, &bn);
        for (uint64_t t = 0; t < T; t++) {
            int32_t id = (int32_t)(g * T + t);
            if (chunk == 0) {
                uint64_t s, cnt;
                orc_static_nochunk(bn, T, t, &s, &cnt);
                for (uint64_t i = 0; i < cnt; i++) owner[bs + s + i] = id;
            } else {
                for (uint64_t j = t; j * chunk < bn; j += T) {
                    uint64_t a = j * chunk;
                    uint64_t e = (bn - a > chunk) ? a + chunk : bn;
                    for (uint64_t i = a; i < e; i++) owner[bs + i] = id;
                }
            }
        }
    }
    return ORC_OK;
}

/*
 * C3 with dist_schedule(static, d) at the team level: distribute chunk
 * j = [j*d, min((j+1)*d, n)) belongs to team j mod G; inside each distribute
 * chunk the team's threads split it by C1 (chunk 0) or C2 (chunk c), the
 * chunk numbering restarting at the distribute chunk's start.  With d = T
 * and c = 1 this is iteration i -> team (i / T) mod G, thread i mod T.
 */
int orc_owner_map_dist(uint64_t n, uint64_t G, uint64_t T, uint64_t d, uint64_t chunk,
                       int32_t *owner)
{
    if (G == 0 || T == 0 || d == 0) return ORC_EINVAL;
    for (uint64_t j = 0; j * d < n; j++) {
        uint64_t g = j % G;
        uint64_t bs = j * d;
        uint64_t bn = (n - bs > d) ? d : n - bs;
        for (uint64_t t = 0; t < T; t++) {
            int32_t id = (int32_t)(g * T + t);
            if (chunk == 0) {
                uint64_t s, cnt;
                orc_static_nochunk(bn, T, t, &s, &cnt);
                for (uint64_t i = 0; i < cnt; i++) owner[bs + s + i] = id;
            } else {
                for (uint64_t k = t; k * chunk < bn; k += T) {
                    uint64_t a = k * chunk;
                    uint64_t e = (bn - a > chunk) ? a + chunk : bn;
                    for (uint64_t i = a; i < e; i++) owner[bs + i] = id;
                }
            }
        }
    }
    return ORC_OK;
}

/*
 * schedule(guided, c) within one team block of bn iterations and T threads.
 * Reading: each request takes max(c, ceil(r / (2T))) of the r iterations not
 * yet handed out, but never more than r.  The sizes depend only on r, so the
 * partition into chunks is the same on every run; only the thread that gets
 * each chunk varies.  Writes the chunk starts in hand-out order (at most
 * max_chunks) and returns their number.
 */
uint64_t orc_guided_chunks(uint64_t bn, uint64_t T, uint64_t c, uint64_t *starts,
                           uint64_t max_chunks)
{
    uint64_t next = 0, k = 0;
    if (c == 0) c = 1;
    while (next < bn) {
        uint64_t r = bn - next;
        uint64_t want = (r + 2 * T - 1) / (2 * T);
        uint64_t size = want > c ? want : c;
        if (size > r) size = r;
        if (k < max_chunks) starts[k] = next;
        k++;
        next += size;
    }
    return k;
}

/* ------------------------------------------------------------------ */
/* loop bodies (C6)                                                    */
/* ------------------------------------------------------------------ */

/* y[i] = alpha*x[i] + y[i] in int32 with two's-complement wrap. */
void orc_axpy_i32(uint64_t n, int32_t alpha, const int32_t *x, int32_t *y)
{
    for (uint64_t i = 0; i < n; i++)
        y[i] = (int32_t)((uint32_t)alpha * (uint32_t)x[i] + (uint32_t)y[i]);
}

/* y[i] = fma(alpha, x[i], y[i]) in fp32, rounded once. */
void orc_axpy_f32(uint64_t n, float alpha, const float *x, float *y)
{
    for (uint64_t i = 0; i < n; i++) y[i] = fmaf(alpha, x[i], y[i]);
}

/* 1-D 3-point stencil, out of place: interior
 * out[i] = fma(c1, in[i-1] + in[i+1], c0*in[i]); the two end points copy in. */
void orc_stencil1d3_f32(uint64_t n, float c0, float c1, const float *in, float *out)
{
    for (uint64_t i = 0; i < n; i++) {
        if (i == 0 || i + 1 == n) {
            out[i] = in[i];
        } else {
            float nb = in[i - 1] + in[i + 1];
            float ce = c0 * in[i];
            out[i] = fmaf(c1, nb, ce);
        }
    }
}

/* 2-D 5-point stencil on an ny x nx row-major grid, out of place: interior
 * out = fma(c1, (north + south) + (east + west), c0*centre); the boundary
 * rows and columns copy in. */
void orc_stencil2d5_f32(uint64_t nx, uint64_t ny, float c0, float c1,
                        const float *in, float *out)
{
    for (uint64_t r = 0; r < ny; r++) {
        for (uint64_t c = 0; c < nx; c++) {
            uint64_t i = r * nx + c;
            if (r == 0 || c == 0 || r + 1 == ny || c + 1 == nx) {
                out[i] = in[i];
            } else {
                float ns = in[i - nx] + in[i + nx];
                float ew = in[i + 1] + in[i - 1];
                float ce = c0 * in[i];
                out[i] = fmaf(c1, ns + ew, ce);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* reductions (C7)                                                     */
/* ------------------------------------------------------------------ */

/* Integer sums: exact modulo 2^64. */
int64_t orc_sum_i64(uint64_t n, const int64_t *a)
{
    uint64_t s = 0;
    for (uint64_t i = 0; i < n; i++) s += (uint64_t)a[i];
    return (int64_t)s;
}

int64_t orc_sum_i32(uint64_t n, const int32_t *a)
{
    uint64_t s = 0;
    for (uint64_t i = 0; i < n; i++) s += (uint64_t)(int64_t)a[i];
    return (int64_t)s;
}

/* max / min over fp32 (no NaN in the inputs; NaN would be skipped). */
double orc_max_f32(uint64_t n, const float *a)
{
    double m = -INFINITY;
    for (uint64_t i = 0; i < n; i++)
        if (a[i] > m) m = a[i];
    return m;
}

double orc_min_f32(uint64_t n, const float *a)
{
    double m = INFINITY;
    for (uint64_t i = 0; i < n; i++)
        if (a[i] < m) m = a[i];
    return m;
}

int64_t orc_max_i64(uint64_t n, const int64_t *a)
{
    int64_t m = INT64_MIN;
    for (uint64_t i = 0; i < n; i++)
        if (a[i] > m) m = a[i];
    return m;
}

int64_t orc_min_i64(uint64_t n, const int64_t *a)
{
    int64_t m = INT64_MAX;
    for (uint64_t i = 0; i < n; i++)
        if (a[i] < m) m = a[i];
    return m;
}

/* int32 data reduce into the int64 result the entry point writes; an empty
 * loop gives the identity of that result type (OpenMP's max / min
 * initializer: the least / greatest value of the reduction item's type). */
int64_t orc_max_i32(uint64_t n, const int32_t *a)
{
    int64_t m = INT64_MIN;
    for (uint64_t i = 0; i < n; i++)
        if (a[i] > m) m = a[i];
    return m;
}

int64_t orc_min_i32(uint64_t n, const int32_t *a)
{
    int64_t m = INT64_MAX;
    for (uint64_t i = 0; i < n; i++)
        if (a[i] < m) m = a[i];
    return m;
}

/*
 * Exact floating-point sum: a long fixed-point accumulator in the manner of
 * Kulisch (U. Kulisch, "Computer Arithmetic and Validity", 2008).  Every
 * addend is a double whose value is an exact fp32 value, bf16 value or
 * product of two fp32 values; the accumulator holds the exact sum and it is
 * rounded once, to nearest-even double.  Digit k (32 bits) has weight
 * 2^(32k + KL_EMIN); each digit is an int64 so that carries may be deferred.
 * Range: the smallest bit of any addend is 2^-350 (product of two fp32
 * subnormals, 2^-298, spelled as a 53-bit significand); the largest addend
 * is below 2^256, and 2^40 of them stay below 2^296 < 2^(32*KL_N + KL_EMIN).
 */
#define KL_N 24
#define KL_EMIN (-352)

typedef struct {
    int64_t d[KL_N];
    uint64_t pending;
} orc_kulisch;

static void kl_init(orc_kulisch *a) { memset(a, 0, sizeof(*a)); }

static void kl_carry(orc_kulisch *a)
{
    for (int k = 0; k < KL_N - 1; k++) {
        int64_t c = a->d[k] >> 32;            /* floor division by 2^32 */
        a->d[k] -= (int64_t)((uint64_t)c << 32);
        a->d[k + 1] += c;
    }
    a->pending = 0;
}

static void kl_add(orc_kulisch *a, double v)
{
    if (v == 0.0) return;
    int ex;
    double f = frexp(fabs(v), &ex);             /* |v| = f * 2^ex, f in [0.5,1) */
    uint64_t m = (uint64_t)ldexp(f, 53);        /* exact 53-bit integer */
    int e = ex - 53;                            /* |v| = m * 2^e */
    int p = e - KL_EMIN;
    if (p < 0 || p / 32 + 2 >= KL_N) abort();   /* outside the stated range */
    int k = p >> 5, sh = p & 31;
    uint64_t lo = m << sh;
    uint64_t hi = sh ? (m >> (64 - sh)) : 0;
    int64_t d0 = (int64_t)(lo & 0xffffffffu), d1 = (int64_t)(lo >> 32), d2 = (int64_t)hi;
    if (v < 0) { d0 = -d0; d1 = -d1; d2 = -d2; }
    a->d[k] += d0;
    a->d[k + 1] += d1;
    a->d[k + 2] += d2;
    if (++a->pending >= (1u << 29)) kl_carry(a);
}

/* bit p of the (non-negative, carried) fixed-point integer */
static int kl_bit(const orc_kulisch *a, int p)
{
    if (p < 0) return 0;
    return (int)(((uint64_t)a->d[p >> 5] >> (p & 31)) & 1u);
}

/* Round the exact accumulated value to the nearest double, ties to even. */
static double kl_round(orc_kulisch *a)
{
    kl_carry(a);
    int neg = a->d[KL_N - 1] < 0;
    if (neg) {
        for (int k = 0; k < KL_N; k++) a->d[k] = -a->d[k];
        kl_carry(a);
    }
    /* now every digit is in [0, 2^32) and the value is non-negative */
    int msb = -1;
    for (int p = 32 * KL_N - 1; p >= 0; p--)
        if (kl_bit(a, p)) { msb = p; break; }
    if (msb < 0) return 0.0;
    /* 64-bit window of bits msb .. msb-63, and a sticky bit for the rest */
    uint64_t win = 0;
    for (int j = 0; j < 64; j++) win = (win << 1) | (uint64_t)kl_bit(a, msb - j);
    int sticky = 0;
    for (int p = msb - 64; p >= 0; p--)
        if (kl_bit(a, p)) { sticky = 1; break; }
    /* window bit 0 has weight 2^(msb - 63 + KL_EMIN) */
    uint64_t mant = win >> 11;                   /* the leading 53 bits */
    uint64_t rem = win & 0x7ff;                  /* the next 11 bits */
    if (rem > 0x400 || (rem == 0x400 && (sticky || (mant & 1)))) mant++;
    double r = ldexp((double)mant, msb - 63 + 11 + KL_EMIN);
    return neg ? -r : r;
}

double orc_exact_sum_f32(uint64_t n, const float *a)
{
    orc_kulisch acc;
    kl_init(&acc);
    for (uint64_t i = 0; i < n; i++) kl_add(&acc, (double)a[i]);
    return kl_round(&acc);
}

/* bf16 values given as their 16-bit patterns (the top half of an fp32). */
double orc_exact_sum_bf16(uint64_t n, const uint16_t *a)
{
    orc_kulisch acc;
    kl_init(&acc);
    for (uint64_t i = 0; i < n; i++) {
        uint32_t bits = (uint32_t)a[i] << 16;
        float f;
        memcpy(&f, &bits, 4);
        kl_add(&acc, (double)f);
    }
    return kl_round(&acc);
}

/* Exact dot product: each fp32 x fp32 product is exact in fp64. */
double orc_exact_dot_f32(uint64_t n, const float *x, const float *y)
{
    orc_kulisch acc;
    kl_init(&acc);
    for (uint64_t i = 0; i < n; i++) kl_add(&acc, (double)x[i] * (double)y[i]);
    return kl_round(&acc);
}

/* Exact sum of arbitrary doubles restricted to the accumulator range; used
 * to combine exact partial sums and by the tests. */
double orc_exact_sum_f64(uint64_t n, const double *a)
{
    orc_kulisch acc;
    kl_init(&acc);
    for (uint64_t i = 0; i < n; i++) kl_add(&acc, a[i]);
    return kl_round(&acc);
}

/* Sum of |a[i]| rounded once (condition-number denominator). */
double orc_exact_abs_sum_f32(uint64_t n, const float *a)
{
    orc_kulisch acc;
    kl_init(&acc);
    for (uint64_t i = 0; i < n; i++) kl_add(&acc, fabs((double)a[i]));
    return kl_round(&acc);
}

/* The exact sum held in an accumulator as a non-overlapping expansion:
 * t_1 = the sum rounded to the nearest double, t_2 = what is left rounded,
 * and so on until nothing is left (each term takes 53 bits off the rest, so a
 * sum of fp32 or bf16 values needs a handful).  Writes at most cap terms and
 * returns how many the sum needs.  The terms of disjoint slices, summed by
 * orc_exact_sum_f64, give the exact sum of the whole rounded once: slices can
 * be summed on separate cores without losing exactness. */
static int kl_terms(orc_kulisch *acc, double *out, int cap)
{
    int k = 0;
    for (;;) {
        orc_kulisch tmp = *acc;                 /* kl_round rewrites its argument */
        double r = kl_round(&tmp);
        if (r == 0.0) return k;
        if (k < cap) out[k] = r;
        k++;
        kl_add(acc, -r);                        /* exact: r is a sum of addend bits */
    }
}

int orc_exact_sum_f32_terms(uint64_t n, const float *a, double *out, int cap)
{
    orc_kulisch acc;
    kl_init(&acc);
    for (uint64_t i = 0; i < n; i++) kl_add(&acc, (double)a[i]);
    return kl_terms(&acc, out, cap);
}

int orc_exact_sum_bf16_terms(uint64_t n, const uint16_t *a, double *out, int cap)
{
    orc_kulisch acc;
    kl_init(&acc);
    for (uint64_t i = 0; i < n; i++) {
        uint32_t bits = (uint32_t)a[i] << 16;
        float f;
        memcpy(&f, &bits, 4);
        kl_add(&acc, (double)f);
    }
    return kl_terms(&acc, out, cap);
}

/* Plain FP64 left-to-right loop (each fp32 value widened exactly, one fp64
 * rounding per add): the CPU speed reference of the reduction configuration,
 * not the oracle of a GPU result. */
double orc_plain_sum_f32(uint64_t n, const float *a)
{
    double s = 0.0;
    for (uint64_t i = 0; i < n; i++) s += (double)a[i];
    return s;
}

/* ------------------------------------------------------------------ */
/* atomic inc (Sec. 3.1): { v = x; x = x >= e ? 0 : x + 1; } returns v */
/* ------------------------------------------------------------------ */
uint32_t orc_atomic_inc(uint32_t *x, uint32_t e)
{
    uint32_t v = *x;
    *x = (v >= e) ? 0u : v + 1u;
    return v;
}

/* ------------------------------------------------------------------ */
/* team shared-memory stack (C10)                                      */
/* ------------------------------------------------------------------ */
/*
 * Reading of __kmpc_alloc_shared(bytes) / free (Sec. 2.1, Listing 1; only the
 * signature is given).  One LIFO stack per team of capacity S bytes in the
 * team's shared memory, plus a per-team slice of Q bytes of a global fallback
 * pool, also LIFO.  A request of b bytes takes r = 16*ceil(max(b,1)/16)
 * bytes: from the shared stack if it fits, else from the pool slice if it
 * fits, else it fails (NULL) and sets the out-of-memory bit.  A free must name
 * the most recent live block of its region with the same size; anything else
 * sets the order-violation bit and changes nothing.
 *
 * Trace: nops pairs (kind, arg).  kind 0 = alloc(arg bytes), whose block is
 * remembered in slot number (count of allocs so far); kind 1 = free(block of
 * slot arg).  Output per op (two int64): for alloc (region, offset) with
 * region 0 = shared, 1 = pool, 2 = failed (offset 0); for free (status bits
 * raised by this op, 0).  Returns the OR of all status bits:
 * bit 0 = out of memory, bit 1 = order violation.
 */
#define ORC_STACK_NOMEM 1
#define ORC_STACK_ORDER 2

int64_t orc_stack_replay(uint64_t S, uint64_t Q, uint64_t nops, const int64_t *ops, int64_t *out)
{
    uint64_t top_s = 0, top_q = 0;
    int64_t status = 0;
    uint64_t nalloc = 0;
    int64_t *slot_region = (int64_t *)calloc(nops + 1, sizeof(int64_t));
    uint64_t *slot_off = (uint64_t *)calloc(nops + 1, sizeof(uint64_t));
    uint64_t *slot_size = (uint64_t *)calloc(nops + 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < nops; i++) {
        int64_t kind = ops[2 * i], arg = ops[2 * i + 1];
        if (kind == 0) {
            uint64_t b = (uint64_t)arg;
            uint64_t r = ((b == 0 ? 1 : b) + 15) / 16 * 16;
            int64_t region;
            uint64_t off = 0;
            if (r <= S - top_s && top_s <= S) {
                region = 0; off = top_s; top_s += r;
            } else if (r <= Q - top_q && top_q <= Q) {
                region = 1; off = top_q; top_q += r;
            } else {
                region = 2; status |= ORC_STACK_NOMEM;
            }
            slot_region[nalloc] = region;
            slot_off[nalloc] = off;
            slot_size[nalloc] = r;
            nalloc++;
            out[2 * i] = region;
            out[2 * i + 1] = (int64_t)off;
        } else {
            int64_t bits = 0;
            uint64_t sl = (uint64_t)arg;
            if (sl >= nalloc) {
                bits = ORC_STACK_ORDER;
            } else {
                int64_t region = slot_region[sl];
                uint64_t off = slot_off[sl], r = slot_size[sl];
                if (region == 0 && off + r == top_s) top_s = off;
                else if (region == 1 && off + r == top_q) top_q = off;
                else if (region == 2) bits = 0;  /* free(NULL) is a no-op */
                else bits = ORC_STACK_ORDER;
            }
            status |= bits;
            out[2 * i] = bits;
            out[2 * i + 1] = 0;
        }
    }
    free(slot_region);
    free(slot_off);
    free(slot_size);
    return status;
}

/* ------------------------------------------------------------------ */
/* MLP cost model 16 -> 64 -> 64 -> 12 (C12), FP64                    */
/* ------------------------------------------------------------------ */
/*
 * Parameters, one flat vector: W1[64][16], b1[64], W2[64][64], b2[64],
 * W3[12][64], b3[12] (row-major, W[out][in]).
 * h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3.
 * Loss: mean over the batch and the 12 outputs of (y - target)^2.
 */
#define M_IN 16
#define M_H 64
#define M_OUT 12
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + M_H * M_IN)
#define OFF_W2 (OFF_B1 + M_H)
#define OFF_B2 (OFF_W2 + M_H * M_H)
#define OFF_W3 (OFF_B2 + M_H)
#define OFF_B3 (OFF_W3 + M_OUT * M_H)
#define M_NPARAM (OFF_B3 + M_OUT)

int orc_mlp_nparam(void) { return M_NPARAM; }

static void mlp_layer(const double *W, const double *b, const double *in, int nin,
                      int nout, int relu, double *out)
{
    for (int o = 0; o < nout; o++) {
        double s = b[o];
        for (int i = 0; i < nin; i++) s += W[o * nin + i] * in[i];
        out[o] = (relu && s < 0.0) ? 0.0 : s;
    }
}

/* forward for a batch: X [B][16] -> Y [B][12] */
void orc_mlp_forward(const double *p, uint64_t B, const double *X, double *Y)
{
    double h1[M_H], h2[M_H];
    for (uint64_t r = 0; r < B; r++) {
        mlp_layer(p + OFF_W1, p + OFF_B1, X + r * M_IN, M_IN, M_H, 1, h1);
        mlp_layer(p + OFF_W2, p + OFF_B2, h1, M_H, M_H, 1, h2);
        mlp_layer(p + OFF_W3, p + OFF_B3, h2, M_H, M_OUT, 0, Y + r * M_OUT);
    }
}

/* loss and gradient d loss / d p (back-propagation by the chain rule) */
double orc_mlp_loss_grad(const double *p, uint64_t B, const double *X, const double *Yt,
                         double *grad)
{
    memset(grad, 0, sizeof(double) * M_NPARAM);
    double loss = 0.0;
    double scale = 1.0 / ((double)B * M_OUT);
    double h1[M_H], h2[M_H], y[M_OUT], dy[M_OUT], dh2[M_H], dh1[M_H];
    for (uint64_t r = 0; r < B; r++) {
        const double *x = X + r * M_IN;
        mlp_layer(p + OFF_W1, p + OFF_B1, x, M_IN, M_H, 1, h1);
        mlp_layer(p + OFF_W2, p + OFF_B2, h1, M_H, M_H, 1, h2);
        mlp_layer(p + OFF_W3, p + OFF_B3, h2, M_H, M_OUT, 0, y);
        for (int o = 0; o < M_OUT; o++) {
            double d = y[o] - Yt[r * M_OUT + o];
            loss += d * d;
            dy[o] = 2.0 * d * scale;
        }
        /* layer 3 */
        for (int o = 0; o < M_OUT; o++) {
            grad[OFF_B3 + o] += dy[o];
            for (int i = 0; i < M_H; i++) grad[OFF_W3 + o * M_H + i] += dy[o] * h2[i];
        }
        for (int i = 0; i < M_H; i++) {
            double s = 0.0;
            for (int o = 0; o < M_OUT; o++) s += p[OFF_W3 + o * M_H + i] * dy[o];
            dh2[i] = h2[i] > 0.0 ? s : 0.0;
        }
        /* layer 2 */
        for (int o = 0; o < M_H; o++) {
            grad[OFF_B2 + o] += dh2[o];
            for (int i = 0; i < M_H; i++) grad[OFF_W2 + o * M_H + i] += dh2[o] * h1[i];
        }
        for (int i = 0; i < M_H; i++) {
            double s = 0.0;
            for (int o = 0; o < M_H; o++) s += p[OFF_W2 + o * M_H + i] * dh2[o];
            dh1[i] = h1[i] > 0.0 ? s : 0.0;
        }
        /* layer 1 */
        for (int o = 0; o < M_H; o++) {
            grad[OFF_B1 + o] += dh1[o];
            for (int i = 0; i < M_IN; i++) grad[OFF_W1 + o * M_IN + i] += dh1[o] * x[i];
        }
    }
    return loss * scale;
}

/* One Adam step (Kingma & Ba, 2015), bias-corrected, step number t >= 1. */
void orc_adam_step(uint64_t np, double *p, const double *g, double *m, double *v,
                   uint64_t t, double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, (double)t);
    double c2 = 1.0 - pow(b2, (double)t);
    for (uint64_t i = 0; i < np; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
