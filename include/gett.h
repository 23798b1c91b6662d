/*
 * gett.h -- C ABI of the GB300 (sm_103a) xGETT library.
 *
 * The operation is the binary tensor contraction of Hornblad, "BLAS-like
 * Interface for Binary Tensor Contractions" (arXiv 2410.06770):
 *
 *   C[o] <- C[o] + sum over contracted coordinates kappa of A[...] * B[...]
 *
 * (Sec. 2.2, the contraction equation; Sec. 6, Alg. 1 adds every product to
 * the value C already holds, so C is ACCUMULATED into, never overwritten).
 *
 * Argument order and meaning are those of the final interface (Sec. 5.7):
 *
 *   xGETT(RANKA, EXTA, INCA, A,  RANKB, EXTB, INCB, B,
 *         CONTS, CONTA, CONTB, PERM,  INCC, C)
 *
 *   RANKA, RANKB  rank of A / B (>= 0; rank 0 is a scalar).
 *   EXTA, EXTB    extents, one per mode (>= 0).  Host arrays, read during
 *                 the call only; may be NULL when the rank is 0.
 *   INCA, INCB    increments in ELEMENTS (not bytes) between neighbours
 *                 along each mode; may be negative (Sec. 7, negative
 *                 increment tests) or zero (broadcast).  Host arrays.
 *   A, B          DEVICE pointers to the element whose coordinates are all
 *                 zero (the "first used data point", Sec. 5.1); with a
 *                 negative increment the other elements lie below it.
 *                 Read only; A and B may alias each other.
 *   CONTS         number of contracted mode pairs (0 <= CONTS <=
 *                 min(RANKA, RANKB)).
 *   CONTA, CONTB  0-based mode indices; CONTA[t] of A is summed against
 *                 CONTB[t] of B, extents must match.  Host arrays; may be
 *                 NULL when CONTS is 0.  Entries of each list are distinct.
 *   PERM          length r_C = RANKA + RANKB - 2*CONTS.  The free indices
 *                 are A's non-contracted modes in ascending order followed
 *                 by B's; PERM[p] is the 0-based OUTPUT POSITION of free
 *                 index p (Sec. 5.6, the fourth encoding).  Must be a
 *                 permutation of 0..r_C-1.  Host array.
 *   INCC          r_C increments of C in elements, indexed by output
 *                 position (the "array of two values" wording of Sec. 5.7 is
 *                 left over from the matrix stage; Sec. 5.4 generalises LD
 *                 to one increment per mode).  Host array.
 *   C             DEVICE pointer to C's coordinate-zero element; read and
 *                 written.  Elements outside the logical tensor (gaps of a
 *                 sub-tensor) are never touched.
 *
 * Extents of C follow from the arguments: EXTC[PERM[p]] = extent of free
 * index p.  A zero free extent means there is nothing to do; a zero
 * contracted extent adds an empty sum (C unchanged).
 *
 * Types: s = float, d = double, c = interleaved single complex, z =
 * interleaved double complex (Sec. 5, prefixes); complex products are not
 * conjugated.  Extension: sbgett takes bfloat16 A and B and a float C.
 *
 * Errors.  Every entry point returns a gett_status.  GETT_ERR_ARG: an
 * argument is invalid; gett_last_error_arg() then returns its 1-based
 * position (1..14, xerbla style) for the calling thread.  GETT_ERR_ALIAS: C
 * overlaps A or B, or C's layout maps two coordinates to the same element
 * (checked by a sufficient test on sorted increments).  GETT_ERR_UNSUPPORTED:
 * more than GETT_MAX_MODES modes of extent > 1 remain in one class after
 * mode fusion, or one class (A-free, B-free or contracted modes) counts more
 * than 2^62 indices (possible only with broadcast, increment-0, modes).  GETT_ERR_CUDA: a CUDA call failed (gett_last_cuda_error()
 * gives the cudaError_t).  GETT_ERR_NOMEM: the call's device workspace
 * (offset tables, split-K partial tiles, packed operands or residue planes,
 * taken from the stream-ordered pool) could not be allocated.  GETT_ERR_TIMEOUT: a device-side wait exceeded its
 * iteration limit; the kernel gave up and the result is undefined.
 *
 * Synchronous forms (xgett) run on the legacy default stream and return
 * after the contraction finished.  _async forms enqueue on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and return at once; device
 * errors of async calls are reported by gett_device_status().
 *
 * There is no CPU fallback: without a usable CUDA device every call returns
 * GETT_ERR_CUDA.
 */
#ifndef GETT_H
#define GETT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GETT_MAX_RANK 64   /* per tensor, as passed by the caller          */
#define GETT_MAX_MODES 24  /* per M/N/K class after squeezing and fusion   */

typedef enum gett_status {
    GETT_OK = 0,
    GETT_ERR_ARG = -1,
    GETT_ERR_ALIAS = -2,
    GETT_ERR_UNSUPPORTED = -3,
    GETT_ERR_CUDA = -4,
    GETT_ERR_TIMEOUT = -5,
    GETT_ERR_NOMEM = -6
} gett_status;

typedef struct gett_complex_float { float re, im; } gett_complex_float;
typedef struct gett_complex_double { double re, im; } gett_complex_double;

/* ---------------------------------------------------------------------- */
/* Plain xGETT (Sec. 5.7).  Synchronous.                                   */
/* ---------------------------------------------------------------------- */
int sgett(int RANKA, const int64_t *EXTA, const int64_t *INCA, const float *A,
          int RANKB, const int64_t *EXTB, const int64_t *INCB, const float *B,
          int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
          const int64_t *INCC, float *C);
int dgett(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
          int RANKB, const int64_t *EXTB, const int64_t *INCB, const double *B,
          int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
          const int64_t *INCC, double *C);
int cgett(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_float *A,
          int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_float *B,
          int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
          const int64_t *INCC, gett_complex_float *C);
int zgett(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_double *A,
          int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_double *B,
          int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
          const int64_t *INCC, gett_complex_double *C);
/* Extension (no counterpart in the thesis): bfloat16 A and B given as raw
 * 16-bit patterns, float C, products accumulated in float. */
int sbgett(int RANKA, const int64_t *EXTA, const int64_t *INCA, const uint16_t *A,
           int RANKB, const int64_t *EXTB, const int64_t *INCB, const uint16_t *B,
           int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
           const int64_t *INCC, float *C);

/* ---------------------------------------------------------------------- */
/* Stream-ordered forms: same arguments plus a cudaStream_t.               */
/* ---------------------------------------------------------------------- */
int sgett_async(int RANKA, const int64_t *EXTA, const int64_t *INCA, const float *A,
                int RANKB, const int64_t *EXTB, const int64_t *INCB, const float *B,
                int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                const int64_t *INCC, float *C, void *stream);
int dgett_async(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
                int RANKB, const int64_t *EXTB, const int64_t *INCB, const double *B,
                int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                const int64_t *INCC, double *C, void *stream);
int cgett_async(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_float *A,
                int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_float *B,
                int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                const int64_t *INCC, gett_complex_float *C, void *stream);
int zgett_async(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_double *A,
                int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_double *B,
                int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                const int64_t *INCC, gett_complex_double *C, void *stream);
int sbgett_async(int RANKA, const int64_t *EXTA, const int64_t *INCA, const uint16_t *A,
                 int RANKB, const int64_t *EXTB, const int64_t *INCB, const uint16_t *B,
                 int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                 const int64_t *INCC, float *C, void *stream);

/* ---------------------------------------------------------------------- */
/* Extended forms: algorithm / kernel-configuration choice and a report.   */
/* ---------------------------------------------------------------------- */
typedef enum gett_algo {
    GETT_ALGO_DEFAULT = 0,    /* library's choice (native arithmetic)      */
    GETT_ALGO_NATIVE = 1,     /* arithmetic in the operand type            */
    GETT_ALGO_OZAKI_BF16 = 2, /* d/z: split-precision modular form on bf16 */
                              /* tensor cores, fp64 recombination (z: the  */
                              /* real 2x2 block form of the complex sum)   */
    GETT_ALGO_BF16X3 = 3,     /* s/c: fp32 split into 2 bf16 pieces, 3     */
                              /* products on tensor cores                  */
    GETT_ALGO_BF16X6 = 4      /* s/c: 3 bf16 pieces, 6 products            */
} gett_algo;

typedef enum gett_family {
    GETT_FAMILY_AUTO = 0,
    GETT_FAMILY_NOOP = 1,     /* empty output or empty sum                 */
    GETT_FAMILY_DENSE = 2,    /* tiled GETT on CUDA cores (FMA)            */
    GETT_FAMILY_OUTER = 3,    /* streaming: no contracted extent > 1       */
    GETT_FAMILY_REDUCE = 4,   /* streaming: few outputs, long sums         */
    GETT_FAMILY_SKINNY = 5,   /* streaming: a free extent <= 8             */
    GETT_FAMILY_TC = 6        /* tensor-core (tcgen05) GEMM: a bf16 operand */
                              /* whose contracted modes fuse to one of      */
                              /* increment 1 and whose free modes fuse to   */
                              /* one with a pitch of whole 16 bytes (16-byte */
                              /* aligned) is read in place by TMA; other    */
                              /* operands, and the split forms' fp32 pieces, */
                              /* are packed first                           */
} gett_family;

/* Conjugation of complex operands (an option of xGEMM-style interfaces; the
 * thesis's contraction never conjugates, Sec. 5).  conj = 0 is Alg. 1.  With
 * GETT_CONJ_A the sum uses conj(A[...]) in place of A[...], with GETT_CONJ_B
 * conj(B[...]); both may be set.  Ignored for the real types (s, d, sb), where
 * conjugation is the identity.  A conjugated operand is first copied, with
 * its imaginary parts negated, into workspace in the planned order (M * K or
 * N * K elements from the stream-ordered pool: GETT_ERR_NOMEM if it does not
 * fit); the contraction then reads that copy. */
#define GETT_CONJ_A 1
#define GETT_CONJ_B 2

typedef struct gett_options {
    int algo;        /* gett_algo                                          */
    int family;      /* gett_family; AUTO lets the selector decide         */
    int config;      /* kernel configuration id within the family; -1 auto */
    int split_k;     /* DENSE: number of K slices (0 = auto, 1 = none)     */
    int moduli;      /* OZAKI_BF16: number of moduli (0 = auto)            */
    int conj;        /* GETT_CONJ_A | GETT_CONJ_B (complex types), 0 = none */
    int reserved[2];
} gett_options;

typedef struct gett_report {
    int family;      /* family that ran                                    */
    int config;      /* configuration that ran; for GETT_FAMILY_TC without */
                     /* the Ozaki form: bit 0 / bit 1 set when A / B was    */
                     /* read in place by TMA (no packed copy)               */
    int split_k;
    int moduli;
    int nm, nn, nk;  /* modes per class after squeeze + fusion             */
    int selector;    /* 0 heuristic, 1 tuning table, 2 learned model, 3 forced */
    int64_t M, N, K; /* products of the class extents                      */
    double flops;    /* 2*M*N*K real (8*M*N*K complex)                      */
    double time_ms;  /* device time of the call's work on `stream` (CUDA   */
                     /* events around every launch and workspace step of   */
                     /* the call, read after it completed); 0 when nothing */
                     /* was launched                                       */
} gett_report;

void gett_options_init(gett_options *opt);

int sgett_ex(int RANKA, const int64_t *EXTA, const int64_t *INCA, const float *A,
             int RANKB, const int64_t *EXTB, const int64_t *INCB, const float *B,
             int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
             const int64_t *INCC, float *C,
             const gett_options *opt, gett_report *rep, void *stream);
int dgett_ex(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
             int RANKB, const int64_t *EXTB, const int64_t *INCB, const double *B,
             int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
             const int64_t *INCC, double *C,
             const gett_options *opt, gett_report *rep, void *stream);
int cgett_ex(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_float *A,
             int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_float *B,
             int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
             const int64_t *INCC, gett_complex_float *C,
             const gett_options *opt, gett_report *rep, void *stream);
int zgett_ex(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_double *A,
             int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_double *B,
             int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
             const int64_t *INCC, gett_complex_double *C,
             const gett_options *opt, gett_report *rep, void *stream);
int sbgett_ex(int RANKA, const int64_t *EXTA, const int64_t *INCA, const uint16_t *A,
              int RANKB, const int64_t *EXTB, const int64_t *INCB, const uint16_t *B,
              int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
              const int64_t *INCC, float *C,
              const gett_options *opt, gett_report *rep, void *stream);

/* ---------------------------------------------------------------------- */
/* Scaled form: C <- alpha * (A . B) + beta * C.                           */
/* Alg. 1 only accumulates (C <- C + A . B); the scaling follows the       */
/* ALPHA and BETA arguments of xGEMM and xGEMV (Sec. 2.3.1): the product   */
/* is scaled by ALPHA and added to C scaled by BETA.                       */
/*   alpha, beta: host pointers to one value of C's element type (float    */
/*     for s and sb, double for d, {re, im} pairs for c and z), read       */
/*     during the call; NULL -> GETT_ERR_ARG at position 15 / 16.          */
/*   beta == 0: C is written without being read (it may hold NaN or        */
/*     uninitialised values), as in BLAS.                                  */
/*   alpha == 0, or an empty sum (a contracted extent 0): A and B are not  */
/*     read; C <- beta * C (zeros when beta == 0; nothing when beta == 1). */
/*   alpha == 1 and beta == 1 is exactly xgett_ex.                         */
/* Every other argument, the options, the report and the synchronisation  */
/* behave as in xgett_ex (the call returns after completion on `stream`).  */
/* Complex split precision (GETT_ALGO_OZAKI_BF16 on z) with a non-real     */
/* alpha or beta stages the product in workspace (16 bytes per output).    */
/* ---------------------------------------------------------------------- */
int sgett_scaled(int RANKA, const int64_t *EXTA, const int64_t *INCA, const float *A,
                 int RANKB, const int64_t *EXTB, const int64_t *INCB, const float *B,
                 int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                 const int64_t *INCC, float *C, const float *alpha, const float *beta,
                 const gett_options *opt, gett_report *rep, void *stream);
int dgett_scaled(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
                 int RANKB, const int64_t *EXTB, const int64_t *INCB, const double *B,
                 int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                 const int64_t *INCC, double *C, const double *alpha, const double *beta,
                 const gett_options *opt, gett_report *rep, void *stream);
int cgett_scaled(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_float *A,
                 int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_float *B,
                 int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                 const int64_t *INCC, gett_complex_float *C, const gett_complex_float *alpha,
                 const gett_complex_float *beta, const gett_options *opt, gett_report *rep, void *stream);
int zgett_scaled(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_double *A,
                 int RANKB, const int64_t *EXTB, const int64_t *INCB, const gett_complex_double *B,
                 int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                 const int64_t *INCC, gett_complex_double *C, const gett_complex_double *alpha,
                 const gett_complex_double *beta, const gett_options *opt, gett_report *rep, void *stream);
int sbgett_scaled(int RANKA, const int64_t *EXTA, const int64_t *INCA, const uint16_t *A,
                  int RANKB, const int64_t *EXTB, const int64_t *INCB, const uint16_t *B,
                  int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                  const int64_t *INCC, float *C, const float *alpha, const float *beta,
                  const gett_options *opt, gett_report *rep, void *stream);

/* ---------------------------------------------------------------------- */
/* Transpose and reduction.  The thesis lists both among the operations a  */
/* full BLAS-like tensor interface would need next (Sec. 9, future work);  */
/* their arguments follow xGETT's conventions (Secs. 5.4-5.7: extents and  */
/* increments per mode, 0-based mode indices, PERM[p] = output position of */
/* free mode p, one INCC per output mode, negative increments point at     */
/* coordinate 0) and the scaled form above (alpha, beta host pointers;     */
/* beta == 0 does not read C; alpha == 0 does not read A).  Both return    */
/* after completion on `stream` and report errors like xgett_ex.           */
/*                                                                         */
/* xGETP: C[o_0 .. o_{r-1} placed by PERM] <- alpha * A[o] + beta * C.     */
/*   Positions: 1 RANKA, 2 EXTA, 3 INCA, 4 A, 5 PERM (RANKA entries),      */
/*   6 INCC, 7 C, 8 alpha, 9 beta.  It equals xGETT with a rank-0 B of     */
/*   value 1 (CONTS = 0).                                                  */
/* xGETR: C[free modes of A, ascending, placed by PERM] <- alpha * sum     */
/*   over the NRED modes RED[0..NRED-1] of A + beta * C.  Positions: 1-4   */
/*   as above, 5 NRED (0..RANKA), 6 RED (distinct modes of A), 7 PERM      */
/*   (RANKA - NRED entries), 8 INCC, 9 C, 10 alpha, 11 beta.  It equals    */
/*   xGETT with B a tensor of ones over the reduced modes; the same        */
/*   selector and kernels run it.                                          */
/* ---------------------------------------------------------------------- */
int sgetp(int RANKA, const int64_t *EXTA, const int64_t *INCA, const float *A,
          const int *PERM, const int64_t *INCC, float *C, const float *alpha,
          const float *beta, void *stream);
int dgetp(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
          const int *PERM, const int64_t *INCC, double *C, const double *alpha,
          const double *beta, void *stream);
int cgetp(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_float *A,
          const int *PERM, const int64_t *INCC, gett_complex_float *C, const gett_complex_float *alpha,
          const gett_complex_float *beta, void *stream);
int zgetp(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_double *A,
          const int *PERM, const int64_t *INCC, gett_complex_double *C, const gett_complex_double *alpha,
          const gett_complex_double *beta, void *stream);
int sbgetp(int RANKA, const int64_t *EXTA, const int64_t *INCA, const uint16_t *A,
           const int *PERM, const int64_t *INCC, float *C, const float *alpha,
           const float *beta, void *stream);
int sgetr(int RANKA, const int64_t *EXTA, const int64_t *INCA, const float *A,
          int NRED, const int *RED, const int *PERM, const int64_t *INCC, float *C,
          const float *alpha, const float *beta, void *stream);
int dgetr(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
          int NRED, const int *RED, const int *PERM, const int64_t *INCC, double *C,
          const double *alpha, const double *beta, void *stream);
int cgetr(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_float *A,
          int NRED, const int *RED, const int *PERM, const int64_t *INCC, gett_complex_float *C,
          const gett_complex_float *alpha, const gett_complex_float *beta, void *stream);
int zgetr(int RANKA, const int64_t *EXTA, const int64_t *INCA, const gett_complex_double *A,
          int NRED, const int *RED, const int *PERM, const int64_t *INCC, gett_complex_double *C,
          const gett_complex_double *alpha, const gett_complex_double *beta, void *stream);
int sbgetr(int RANKA, const int64_t *EXTA, const int64_t *INCA, const uint16_t *A,
           int NRED, const int *RED, const int *PERM, const int64_t *INCC, float *C,
           const float *alpha, const float *beta, void *stream);

/* ---------------------------------------------------------------------- */
/* Allocation-free double-precision form.  The thesis has no counterpart;  */
/* this entry point exists for callers that must not allocate device       */
/* memory while they run (a process that budgets all device memory up     */
/* front, a latency-critical loop that cannot afford cudaFree's implicit   */
/* device-wide synchronisation, a framework whose own allocator owns the   */
/* device).  Same 14 arguments and semantics as dgett, stream-ordered on   */
/* `stream` like dgett_async, computed by the dense CUDA-core kernel.  Its */
/* scratch (16 * (M + N + K) bytes of offset tables, M, N, K = products of */
/* the free-A, free-B and contracted extents) lives in one fixed 4 MiB     */
/* device array of the library that every GPU loading the library holds    */
/* until the process exits; problems with M + N + K greater than           */
/* GETT_NOALLOC_MAX_INDEX_SUM are rejected with GETT_ERR_UNSUPPORTED and   */
/* nothing is launched.  It calls no cudaMalloc or cudaFree.  The first    */
/* call on a device (with that device current) looks up the array's device */
/* address with cudaGetSymbolAddress; make that first call before any      */
/* stream capture.  All calls share the array (it keeps the last call's    */
/* contents, none of which needs to start at zero): calls whose work       */
/* overlaps on the GPU race and must be ordered by the caller.             */
/* ---------------------------------------------------------------------- */
#define GETT_NOALLOC_MAX_INDEX_SUM 262144
int dgett_noalloc(int RANKA, const int64_t *EXTA, const int64_t *INCA, const double *A,
                  int RANKB, const int64_t *EXTB, const int64_t *INCB, const double *B,
                  int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                  const int64_t *INCC, double *C, void *stream);

/* ---------------------------------------------------------------------- */
/* Planner inspection (host only, no device work).  Validates the 14       */
/* arguments (pointers are not inspected) and describes the canonical      */
/* problem: modes of each class after dropping extent-1 modes, flipping    */
/* negative increments and fusing stride-compatible neighbours.            */
/* ---------------------------------------------------------------------- */
typedef struct gett_plan_info {
    int nm, nn, nk;
    int empty;                              /* nothing to compute          */
    int64_t M, N, K;
    int64_t m_ext[GETT_MAX_MODES], m_inca[GETT_MAX_MODES], m_incc[GETT_MAX_MODES];
    int64_t n_ext[GETT_MAX_MODES], n_incb[GETT_MAX_MODES], n_incc[GETT_MAX_MODES];
    int64_t k_ext[GETT_MAX_MODES], k_inca[GETT_MAX_MODES], k_incb[GETT_MAX_MODES];
    int64_t off_a, off_b, off_c;            /* element offsets from flips   */
} gett_plan_info;

int gett_plan_describe(int RANKA, const int64_t *EXTA, const int64_t *INCA,
                       int RANKB, const int64_t *EXTB, const int64_t *INCB,
                       int CONTS, const int *CONTA, const int *CONTB, const int *PERM,
                       const int64_t *INCC, gett_plan_info *out);

/* ---------------------------------------------------------------------- */
/* Diagnostics.                                                            */
/* ---------------------------------------------------------------------- */
int gett_last_error_arg(void);       /* 1-based argument of last GETT_ERR_ARG */
int gett_last_cuda_error(void);      /* cudaError_t of last GETT_ERR_CUDA     */
const char *gett_status_string(int status);
/* Reads (and clears) the device error word that kernels set when a bounded
 * wait gives up; synchronises the device.  GETT_OK or GETT_ERR_TIMEOUT. */
int gett_device_status(void);
int gett_version(void);              /* major*10000 + minor*100 + patch      */
/* Failure-detection check (no counterpart in the thesis): launches one
 * thread that waits, with a limit of `limit_cycles` SM clock cycles, on a
 * device barrier that nothing completes.  The bounded wait gives up, records
 * its code in the device error word and the kernel returns; the call then
 * reads the word like gett_device_status and returns GETT_ERR_TIMEOUT, with
 * the CUDA context still usable.  Synchronous. */
int gett_check_wait_timeout(long long limit_cycles);

/* Parameters of the split-precision form GETT_ALGO_OZAKI_BF16 for a
 * contraction with K summed terms (the modular form of the Ozaki scheme,
 * Ozaki, Uchino and Imamura 2025; the thesis names no split method).  Host
 * only: no device work.  moduli_wanted = 0 picks the smallest count whose
 * product P leaves at least 50 bits a operand; counts below 2 are raised to
 * 2.  *L receives the count, *bits the bits each operand's scaled integers
 * keep (the largest b <= 52 with K * 2^(2b) < P / 2, so the exact sum is
 * recovered from its residues), and moduli[0..L) (if not NULL, at least
 * GETT_OZAKI_MAX_MODULI entries) the odd, pairwise coprime moduli, each at
 * most 255 so that symmetric residues are exact in bfloat16.  A complex
 * contraction sums 2K real products (pass 2K).  GETT_ERR_ARG: K < 0,
 * moduli_wanted outside [0, GETT_OZAKI_MAX_MODULI], L or bits NULL. */
#define GETT_OZAKI_MAX_MODULI 20
int gett_ozaki_params(int64_t K, int moduli_wanted, int *L, int *bits, int *moduli);

#ifdef __cplusplus
}
#endif

#endif /* GETT_H */
