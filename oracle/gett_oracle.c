/*
 * gett_oracle.c -- plain, slow CPU oracle for the binary tensor contraction
 * xGETT (thesis "BLAS-like Interface for Binary Tensor Contractions",
 * Hornblad 2024, arXiv 2410.06770).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  The CUDA
 * library never calls it and shares no code, header or helper with it.
 *
 * What it computes (Sec. 2.2, the contraction equation; Sec. 6, Alg. 1):
 *   for every output coordinate o:
 *     C[sum_q o_q INCC[q]] <- C[...] + sum_kappa A[...] * B[...]
 *   where the free modes are A's non-contracted modes in ascending order
 *   followed by B's (Sec. 5.6, option 4 of the PERM encodings), free index p
 *   is placed at output position PERM[p], and kappa runs over the contracted
 *   coordinates with the first contracted index fastest (Alg. 2).
 *
 * Evaluation order follows Alg. 1 literally: each product is added to the
 * current C element in sequence, starting from the value C already holds
 * (C is accumulated into, never zeroed).  Build with -ffp-contract=off so no
 * multiply-add is fused and the result is deterministic.
 *
 * Readings of the thesis taken here (all listed in the design notes):
 *  - PERM[p] is the OUTPUT POSITION of free index p (Sec. 5.6: "the integers
 *    written in each position ... represent the placement").
 *  - INCC has one entry per output mode (Sec. 5.4 generalises LD to INC; the
 *    "array of two values" wording is left over from the matrix stage).
 *  - In Alg. 1 the contracted loop uses the contracted-mode increments
 *    IncContA/IncContB, and the two IncCoords calls take ExtContInd for the
 *    contracted coordinates and ExtFreeInd for the free ones (the printed
 *    arguments are swapped).
 *  - Indices are 0-based (the interface is C).
 *  - Pointers address the element whose coordinates are all zero ("first used
 *    data point"); negative increments reach lower addresses.
 *  - An empty index list gives one iteration (rank-0 tensors are scalars);
 *    a zero extent gives none.
 *
 * Parity pins: tests/test_oracle_pins.py (GEMM/GEMV/DOT/GER reductions against
 * numpy BLAS, integer-exact comparison with numpy.einsum, the coordinate
 * order printed in Sec. 6, the layout figures with increments [1,3,9] and
 * [1,5,25], permutation/commutativity/stride invariance, brute force).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* Alg. 2 (IncCoords): odometer increment, first coordinate fastest.       */
/* Returns at once when there are no indices.                              */
/* ---------------------------------------------------------------------- */
static void inc_coords(int num_of_ind, int64_t *coords, const int64_t *exts)
{
    if (num_of_ind <= 0) return;
    int i = 0;
    do {
        coords[i] = (coords[i] + 1) % exts[i];
        i = i + 1;
    } while (coords[i - 1] == 0 && i < num_of_ind);
}

/* Exported so the tests can compare the visiting order with the sequence
 * printed in Sec. 6 ([0,0,0], [1,0,0], [2,0,0], [0,1,0], ...). */
void oracle_inc_coords(int num_of_ind, int64_t *coords, const int64_t *exts)
{
    inc_coords(num_of_ind, coords, exts);
}

/* ---------------------------------------------------------------------- */
/* Preprocessing of Sec. 6: the arrays Alg. 1 works on.                    */
/* ---------------------------------------------------------------------- */
typedef struct {
    int num_free;          /* NumFreeInd  = RANKA + RANKB - 2*CONTS        */
    int num_cont;          /* NumContInd  = CONTS                          */
    int64_t size_free;     /* SizeFreeInd = prod ExtFreeInd (1 if none)    */
    int64_t size_cont;     /* SizeContInd = prod ExtContInd (1 if none)    */
    int64_t *ext_free;     /* ExtFreeInd[q], ordered by output position q  */
    int64_t *inc_c;        /* IncC[q]                                      */
    int64_t *inc_free;     /* IncFreeInd[q]: increment in the owning tensor */
    int *ten_free;         /* TenFreeInd[q]: 0 = A, 1 = B                  */
    int64_t *ext_cont;     /* ExtContInd[t]                                */
    int64_t *inc_cont_a;   /* IncContA[t] = INCA[CONTA[t]]                 */
    int64_t *inc_cont_b;   /* IncContB[t] = INCB[CONTB[t]]                 */
} prep_t;

static void prep_free(prep_t *p)
{
    free(p->ext_free); free(p->inc_c); free(p->inc_free); free(p->ten_free);
    free(p->ext_cont); free(p->inc_cont_a); free(p->inc_cont_b);
}

/* Returns 0 on success, a negative number when the arguments do not describe
 * a valid contraction (the oracle only checks what it needs to index safely). */
static int prepare(prep_t *p,
                   int RANKA, const int64_t *EXTA, const int64_t *INCA,
                   int RANKB, const int64_t *EXTB, const int64_t *INCB,
                   int CONTS, const int *CONTA, const int *CONTB,
                   const int *PERM, const int64_t *INCC)
{
    memset(p, 0, sizeof(*p));
    if (RANKA < 0 || RANKB < 0 || CONTS < 0 || CONTS > RANKA || CONTS > RANKB)
        return -1;
    int nf = RANKA + RANKB - 2 * CONTS;
    p->num_free = nf;
    p->num_cont = CONTS;
    int nalloc_f = nf > 0 ? nf : 1, nalloc_c = CONTS > 0 ? CONTS : 1;
    p->ext_free = calloc(nalloc_f, sizeof(int64_t));
    p->inc_c = calloc(nalloc_f, sizeof(int64_t));
    p->inc_free = calloc(nalloc_f, sizeof(int64_t));
    p->ten_free = calloc(nalloc_f, sizeof(int));
    p->ext_cont = calloc(nalloc_c, sizeof(int64_t));
    p->inc_cont_a = calloc(nalloc_c, sizeof(int64_t));
    p->inc_cont_b = calloc(nalloc_c, sizeof(int64_t));
    char *is_cont_a = calloc(RANKA > 0 ? RANKA : 1, 1);
    char *is_cont_b = calloc(RANKB > 0 ? RANKB : 1, 1);
    char *placed = calloc(nalloc_f, 1);
    int rc = 0;

    for (int t = 0; t < CONTS; ++t) {
        int ma = CONTA[t], mb = CONTB[t];
        if (ma < 0 || ma >= RANKA || mb < 0 || mb >= RANKB ||
            is_cont_a[ma] || is_cont_b[mb] || EXTA[ma] != EXTB[mb]) { rc = -2; goto done; }
        is_cont_a[ma] = 1; is_cont_b[mb] = 1;
        p->ext_cont[t] = EXTA[ma];
        p->inc_cont_a[t] = INCA[ma];
        p->inc_cont_b[t] = INCB[mb];
    }
    /* Free index p: A's free modes ascending, then B's (Sec. 5.6). */
    int fp = 0;
    for (int tensor = 0; tensor < 2; ++tensor) {
        int rank = tensor == 0 ? RANKA : RANKB;
        const int64_t *ext = tensor == 0 ? EXTA : EXTB;
        const int64_t *inc = tensor == 0 ? INCA : INCB;
        const char *is_cont = tensor == 0 ? is_cont_a : is_cont_b;
        for (int mode = 0; mode < rank; ++mode) {
            if (is_cont[mode]) continue;
            int q = PERM[fp];
            if (q < 0 || q >= nf || placed[q]) { rc = -3; goto done; }
            placed[q] = 1;
            p->ext_free[q] = ext[mode];
            p->inc_free[q] = inc[mode];
            p->ten_free[q] = tensor;
            p->inc_c[q] = INCC[q];
            ++fp;
        }
    }
    p->size_free = 1;
    for (int q = 0; q < nf; ++q) p->size_free *= p->ext_free[q];
    p->size_cont = 1;
    for (int t = 0; t < CONTS; ++t) p->size_cont *= p->ext_cont[t];
done:
    free(is_cont_a); free(is_cont_b); free(placed);
    if (rc) prep_free(p);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Alg. 1, generated for each element type.  The free-index range can be   */
/* split into chunks [i0, i1); a chunk starts from the free coordinates of  */
/* its first position (mixed-radix decode, first coordinate fastest, the    */
/* same sequence IncCoords walks) and then continues with IncCoords.  Every */
/* output element therefore sees exactly the same sequence of additions     */
/* whatever the chunking, and chunks may run in parallel when C's layout is */
/* injective.                                                               */
/* ---------------------------------------------------------------------- */
#define DEFINE_ALG1(NAME, T, ACC, LOADC, STOREC, MAC)                           \
static void NAME(const prep_t *p, const T *A, const T *B, T *C,                 \
                 int64_t i0, int64_t i1)                                        \
{                                                                               \
    int nf = p->num_free, nc = p->num_cont;                                     \
    int64_t coord_free[64], coord_cont[64];                                     \
    int64_t r = i0;                                                             \
    if (i0 >= i1) return;                                                       \
    for (int q = 0; q < nf; ++q) {                                              \
        coord_free[q] = r % p->ext_free[q];                                     \
        r /= p->ext_free[q];                                                    \
    }                                                                           \
    for (int64_t i = i0; i < i1; ++i) {                                         \
        int64_t idx_c = 0, free_idx_a = 0, free_idx_b = 0;                      \
        for (int j = 0; j < nf; ++j) {                                          \
            idx_c += p->inc_c[j] * coord_free[j];                               \
            if (p->ten_free[j] == 0)                                            \
                free_idx_a += p->inc_free[j] * coord_free[j];                   \
            else                                                                \
                free_idx_b += p->inc_free[j] * coord_free[j];                   \
        }                                                                       \
        for (int t = 0; t < nc; ++t) coord_cont[t] = 0;                         \
        ACC acc = LOADC(C[idx_c]);                                              \
        for (int64_t j = 0; j < p->size_cont; ++j) {                            \
            int64_t idx_a = free_idx_a, idx_b = free_idx_b;                     \
            for (int k = 0; k < nc; ++k) {                                      \
                idx_a += p->inc_cont_a[k] * coord_cont[k];                      \
                idx_b += p->inc_cont_b[k] * coord_cont[k];                      \
            }                                                                   \
            MAC(acc, A[idx_a], B[idx_b]);                                       \
            inc_coords(nc, coord_cont, p->ext_cont);                            \
        }                                                                       \
        STOREC(C[idx_c], acc);                                                  \
        inc_coords(nf, coord_free, p->ext_free);                                \
    }                                                                           \
}

/* real double: C <- C + A*B in double, one rounding per multiply and add */
#define LOAD_SAME(x) (x)
#define STORE_SAME(dst, v) ((dst) = (v))
#define MAC_REAL(acc, a, b) ((acc) = (acc) + (a) * (b))
DEFINE_ALG1(alg1_f64, double, double, LOAD_SAME, STORE_SAME, MAC_REAL)

/* real, accumulated in long double and rounded to double once at the end
 * (binary128 on aarch64 hosts, x87 80-bit on x86_64 hosts) */
#define LOAD_LD(x) ((long double)(x))
#define STORE_LD(dst, v) ((dst) = (double)(v))
#define MAC_LD(acc, a, b) ((acc) = (acc) + (long double)(a) * (long double)(b))
DEFINE_ALG1(alg1_f64_ld, double, long double, LOAD_LD, STORE_LD, MAC_LD)

/* complex double, interleaved (re, im), no conjugation:
 * (ar + i ai)(br + i bi) = (ar br - ai bi) + i (ar bi + ai br) */
typedef struct { double re, im; } zdouble;
static inline zdouble zload(zdouble x) { return x; }
#define STORE_Z(dst, v) ((dst) = (v))
#define MAC_Z(acc, a, b) do {                                   \
        double pr = (a).re * (b).re - (a).im * (b).im;          \
        double pi = (a).re * (b).im + (a).im * (b).re;          \
        (acc).re = (acc).re + pr;                               \
        (acc).im = (acc).im + pi;                               \
    } while (0)
DEFINE_ALG1(alg1_z, zdouble, zdouble, zload, STORE_Z, MAC_Z)

#define DEFINE_ENTRY(NAME, T, ALG)                                               \
int NAME(int RANKA, const int64_t *EXTA, const int64_t *INCA, const T *A,        \
         int RANKB, const int64_t *EXTB, const int64_t *INCB, const T *B,        \
         int CONTS, const int *CONTA, const int *CONTB, const int *PERM,         \
         const int64_t *INCC, T *C, int nthreads)                                \
{                                                                                \
    prep_t p;                                                                    \
    int rc = prepare(&p, RANKA, EXTA, INCA, RANKB, EXTB, INCB,                   \
                     CONTS, CONTA, CONTB, PERM, INCC);                           \
    if (rc) return rc;                                                           \
    if (p.num_free > 64 || p.num_cont > 64) { prep_free(&p); return -4; }        \
    int64_t n = p.size_free;                                                     \
    if (nthreads <= 1 || n < 2) {                                                \
        ALG(&p, A, B, C, 0, n);                                                  \
    } else {                                                                     \
        int64_t nchunks = (int64_t)nthreads * 8;                                 \
        if (nchunks > n) nchunks = n;                                            \
        _Pragma("omp parallel for schedule(dynamic, 1) num_threads(nthreads)")   \
        for (int64_t c = 0; c < nchunks; ++c) {                                  \
            int64_t lo = n * c / nchunks, hi = n * (c + 1) / nchunks;            \
            ALG(&p, A, B, C, lo, hi);                                            \
        }                                                                        \
    }                                                                            \
    prep_free(&p);                                                               \
    return 0;                                                                    \
}

/* nthreads <= 1: the single-threaded Alg. 1 exactly as printed.
 * nthreads > 1: output positions split over threads (requires injective C). */
DEFINE_ENTRY(oracle_dgett, double, alg1_f64)
DEFINE_ENTRY(oracle_dgett_ld, double, alg1_f64_ld)
DEFINE_ENTRY(oracle_zgett, zdouble, alg1_z)

/* ---------------------------------------------------------------------- */
/* Second, independent oracle for brute-force cross-checks on tiny inputs. */
/* No preprocessing arrays and no odometer: every output element is found  */
/* by decoding a flat index over the OUTPUT modes directly, and each       */
/* contracted coordinate tuple by decoding a flat index over CONTA order.  */
/* The free mode at output position q is located by searching PERM.        */
/* Same summation order (first contracted index fastest), so on the same    */
/* inputs it must agree with oracle_dgett bit for bit.                      */
/* ---------------------------------------------------------------------- */
int oracle_dgett_direct(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
                        int RANKB, const int64_t *EXTB, const int64_t *INCB, const double *B,
                        int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                        const int64_t *INCC, double *C)
{
    int nf = RANKA + RANKB - 2 * CONTS;
    if (nf < 0 || nf > 64 || CONTS > 64) return -1;
    /* which tensor/mode feeds output position q */
    int src_tensor[64], src_mode[64];
    int fp = 0;
    for (int m = 0; m < RANKA; ++m) {
        int contracted = 0;
        for (int t = 0; t < CONTS; ++t) if (CONTA[t] == m) contracted = 1;
        if (contracted) continue;
        src_tensor[PERM[fp]] = 0; src_mode[PERM[fp]] = m; ++fp;
    }
    for (int m = 0; m < RANKB; ++m) {
        int contracted = 0;
        for (int t = 0; t < CONTS; ++t) if (CONTB[t] == m) contracted = 1;
        if (contracted) continue;
        src_tensor[PERM[fp]] = 1; src_mode[PERM[fp]] = m; ++fp;
    }
    int64_t nout = 1;
    for (int q = 0; q < nf; ++q)
        nout *= src_tensor[q] == 0 ? EXTA[src_mode[q]] : EXTB[src_mode[q]];
    int64_t ncont = 1;
    for (int t = 0; t < CONTS; ++t) ncont *= EXTA[CONTA[t]];
    for (int64_t flat = 0; flat < nout; ++flat) {
        int64_t oc = 0, oa = 0, ob = 0, r = flat;
        for (int q = 0; q < nf; ++q) {
            int64_t e = src_tensor[q] == 0 ? EXTA[src_mode[q]] : EXTB[src_mode[q]];
            int64_t x = r % e;
            r /= e;
            oc += x * INCC[q];
            if (src_tensor[q] == 0) oa += x * INCA[src_mode[q]];
            else ob += x * INCB[src_mode[q]];
        }
        double acc = C[oc];
        for (int64_t kflat = 0; kflat < ncont; ++kflat) {
            int64_t ia = oa, ib = ob, rk = kflat;
            for (int t = 0; t < CONTS; ++t) {
                int64_t e = EXTA[CONTA[t]];
                int64_t x = rk % e;
                rk /= e;
                ia += x * INCA[CONTA[t]];
                ib += x * INCB[CONTB[t]];
            }
            acc = acc + A[ia] * B[ib];
        }
        C[oc] = acc;
    }
    return 0;
}

/* Size of long double in bits of significand, so reports can state which
 * "long double" the extended oracle used on this host. */
int oracle_long_double_mant_dig(void)
{
    return __LDBL_MANT_DIG__;
}
