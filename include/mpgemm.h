/*
 * mpgemm — multiple-precision dense real matrix multiplication C := AB on one
 * NVIDIA GB300 (sm_103a).
 *
 * The operation is the paper's: Kouya, "Tuning Technique for Multiple
 * Precision Dense Matrix Multiplication using Prediction of Computational
 * Time" (arXiv:1710.01839), Section 2: C := AB with A in R^{m x l},
 * B in R^{l x n}, c_ij = sum_{k=1..l} a_ik b_kj (Eq 1), computed by the
 * simple algorithm (Eq 1), the block algorithm with block size n_min (Eq 2)
 * or Strassen's recursion P1..P7 (Eq 3), in double-double (DD), quad-double
 * (QD) or p-bit multi-limb binary floating point (the MPFR stand-in of
 * Section 4.2).
 *
 * Conventions shared by every entry point:
 *   - All matrix pointers are DEVICE pointers owned by the caller.  The
 *     library never frees them.  C must not overlap A or B (MPGEMM_EINVAL).
 *   - Layout: row-major planes.  DD: 2 planes [hi | lo] of rows*cols doubles
 *     (value hi + lo, |lo| <= ulp(hi)/2).  QD: 4 planes x0..x3 (value
 *     x0 + x1 + x2 + x3, non-overlapping).  Multi-limb with p = prec_bits
 *     = 32 w: (2 + w) planes of rows*cols uint32 words: [exponent (int32) |
 *     flags (bit0 sign, bit1 zero) | limb 0 (least significant) .. limb w-1],
 *     value (-1)^sign * M * 2^(exponent - p), M = sum limb_i 2^(32 i) in
 *     [2^(p-1), 2^p); zero has M = 0, exponent 0, flags bit1 set.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream).  Argument errors are returned at once and nothing is
 *     launched.  Errors found on the device (multi-limb exponent overflow, a
 *     bounded wait that gave up) set a per-device status word that
 *     mpgemm_stream_status() reads.
 *   - Return value: MPGEMM_OK (0) or a negative mpgemm_status.
 *   - m, l, n may be 0 (nothing to do, C untouched when m*n == 0; C = 0 when
 *     l == 0).
 */
#ifndef MPGEMM_H
#define MPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPGEMM_SIMPLE = 0,    /* Eq 1: one output per thread, k ascending, no staging        */
    MPGEMM_BLOCK = 1,     /* Eq 2: n_min-blocked, shared-memory staged, register tiled    */
    MPGEMM_STRASSEN = 2,  /* Eq 3: strassen_depth levels of P1..P7, leaves = block(n_min) */
    MPGEMM_AUTO = 3       /* algorithm, n_min and depth from the tuner / cost model       */
} mpgemm_algo;

typedef enum {
    MPGEMM_OK = 0,
    MPGEMM_EINVAL = -1,       /* bad argument (negative size, NULL, overlap, bad n_min)   */
    MPGEMM_EUNSUPPORTED = -2, /* valid but not supported (precision not built, size       */
                              /* beyond a kernel's limits)                                 */
    MPGEMM_ECUDA = -3,        /* a CUDA call failed; mpgemm_last_cuda_error() has it       */
    MPGEMM_EOVERFLOW = -4,    /* device: a multi-limb exponent left the int32 range (or a  */
                              /* conversion to double left the normal double range)        */
    MPGEMM_ETIMEOUT = -5,     /* device: a bounded wait gave up                            */
    MPGEMM_ENOMEM = -6        /* workspace allocation failed or is too small               */
} mpgemm_status;

typedef enum { MPGEMM_KIND_DD = 0, MPGEMM_KIND_QD = 1, MPGEMM_KIND_MP = 2 } mpgemm_kind;

/* ---------------------------------------------------------------------------
 * The GEMM (Section 2, Eqs 1-3).
 *   algo           mpgemm_algo.
 *   n_min          block size of Eq 2 (power of two, 16..256).  On the GPU it is
 *                  the edge of the square C block one CTA computes when
 *                  n_min <= the format's largest CTA tile (64 DD, 32 QD, 16 MP),
 *                  and otherwise the edge of the super-tile of CTAs that run
 *                  back to back (L2 blocking).  <= 0 selects the default.
 *   strassen_depth levels of Eq 3 (0..4) for MPGEMM_STRASSEN.  A dimension
 *                  that 2^depth does not divide is zero-extended to the next
 *                  multiple of 2^depth (A and B are read as if padded with
 *                  zero rows and columns; nothing is copied) and only the
 *                  m x n block of C is written.
 * Strassen needs workspace (mpgemm_workspace_size); it is taken from the
 * buffer given to mpgemm_set_workspace, else allocated stream-ordered
 * (cudaMallocAsync) and released on the same stream.
 * ------------------------------------------------------------------------- */
int mpgemm_dd(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int algo,
              int n_min, int strassen_depth, void* stream);
int mpgemm_qd(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int algo,
              int n_min, int strassen_depth, void* stream);
/* prec_bits = 32 w, w in {1, 2, 4, 8, 16, 32, 64}.  Round to nearest, ties to
   even, after every multiply and every add (c <- RN(c + RN(a b)), k
   ascending); simple and block results are bit-identical to each other. */
int mpgemm_mp(int64_t m, int64_t l, int64_t n, int prec_bits, const uint32_t* A, const uint32_t* B,
              uint32_t* C, int algo, int n_min, int strassen_depth, void* stream);

/* Which kernel runs the block algorithm (and Strassen's leaves) of
 * mpgemm_mp at 512, 1024 and 2048 bits (other widths and the simple
 * algorithm are unaffected):
 *   MPGEMM_MP_LEAF_THREAD  one thread per element of C, the w limbs of every
 *                          value in that thread's registers;
 *   MPGEMM_MP_LEAF_TEAM    a team of w / 8 lanes of a warp per element of C,
 *                          8 limbs per lane; products by operand scanning with
 *                          the partial sums passed between lanes by warp
 *                          shuffles, carries between lanes by a look-ahead on
 *                          warp ballots;
 *   MPGEMM_MP_LEAF_DEFAULT the team kernel when the one-thread kernel's
 *                          grid (16 x 16 elements of C per CTA, times the
 *                          batch) has at most one CTA for every two SMs of
 *                          the stream's partition, else the one-thread kernel.
 * Both kernels keep Eq 1's operation sequence and give the same bits.
 * Process-wide, not tied to a stream: set it between calls.  Returns the
 * previous setting, MPGEMM_EINVAL for any other value. */
typedef enum { MPGEMM_MP_LEAF_DEFAULT = 0, MPGEMM_MP_LEAF_THREAD = 1, MPGEMM_MP_LEAF_TEAM = 2 } mpgemm_mp_leaf;
int mpgemm_set_mp_leaf(int leaf);
/* The kernel (MPGEMM_MP_LEAF_THREAD or _TEAM) a block GEMM of `batch`
 * products of m x n elements at prec_bits uses under the current setting on
 * a stream of `sms` SMs (mpgemm_stream_sms).  Host arithmetic only;
 * MPGEMM_EINVAL for prec_bits not a positive multiple of 32, negative sizes,
 * batch or sms below 1. */
int mpgemm_mp_leaf_choice(int prec_bits, int64_t m, int64_t n, int64_t batch, int sms);

/* ---------------------------------------------------------------------------
 * Split-precision DD GEMM on the INT8 tensor path (an Ozaki-style scheme; the
 * paper has no counterpart, it is an extension of its DD GEMM):
 *   1. e_i = largest frexp exponent of row i of A's hi plane, f_j of column j
 *      of B's hi plane;
 *   2. every element, scaled by 2^-e_i (A) or 2^-f_j (B), is truncated toward
 *      zero to 7 S bits and split into S signed base-128 digits (int8);
 *   3. level sums L_g = sum_{s+t=g} D_s^A D_t^B for g = 2..S+1, exact in int32
 *      (int8 x int8 tensor-core products);
 *   4. c_ij = (RN(x), RN(x - RN(x))) with x = 2^(e_i+f_j) sum_g L_g 2^-7g,
 *      summed exactly.
 * num_slices S in 1..18 (0 = 16).  Error: |C - AB| <= about
 * 2 l 2^-7S max|a'| max|b'| 2^(e_i+f_j) plus the final DD rounding; S = 16
 * gives <= 2^-100 |A||B| for entries within a few binades of their row /
 * column maximum.  Limits: S * 127^2 * l < 2^31, m and n <= 65535.
 * Workspace: mpgemm_ozaki_workspace_size() bytes, from the buffer set with
 * mpgemm_set_workspace or allocated stream-ordered.
 * ------------------------------------------------------------------------- */
int mpgemm_dd_ozaki(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int num_slices,
                    void* stream);
size_t mpgemm_ozaki_workspace_size(int64_t m, int64_t l, int64_t n, int num_slices);
int mpgemm_ozaki_slices_default(void);
/* Steps 1-2 alone: digits of a DD matrix X (rows x cols planes).  by_col = 0:
   row scaling, digits as S planes of rows x lp int8 (lp = cols rounded up to
   128, zero padded); by_col = 1: column scaling, digits transposed as S planes
   of cols x lp (lp = rows rounded up to 128).  expo receives the exponents. */
int mpgemm_ozaki_split(int by_col, int64_t rows, int64_t cols, const double* X, int num_slices, int* expo,
                       signed char* digits, void* stream);
/* Step 3 alone: levels = S planes (g = 2..S+1) of m x n int32 from digit
   planes laid out as mpgemm_ozaki_split writes them. */
int mpgemm_ozaki_levels(int64_t m, int64_t l, int64_t n, int num_slices, const signed char* DA,
                        const signed char* DB, int* levels, void* stream);
/* The same scheme with a choice of digits (digit_kind):
 *   MPGEMM_DIGITS_INT8 (0): base-128 digits in [-127, 127] as int8, products
 *     on mma.sync s8 (what mpgemm_dd_ozaki does; S <= 18, default 16);
 *   MPGEMM_DIGITS_E4M3 (1): each element scaled by 2^-(e_i+1) (one bit of
 *     headroom) is truncated toward zero to 5 S bits and written in balanced
 *     base-32 digits (every digit in [-16, 16], exact in FP8 e4m3), stored as
 *     e4m3 codes; products on the tcgen05 tensor cores (kind::f8f6f4) with
 *     f32 accumulation in tensor memory, exact because every partial sum of
 *     Q = floor(2^24 / (256 lp)) slice pairs is an integer below 2^24 (l <=
 *     65536), moved to int32 after every Q pairs; S <= 24, default 22
 *     (<= 2^-100 |A||B| on the same inputs as 16 int8 slices).  For
 *     mpgemm_ozaki_levels_ex with e4m3 digits, DA and DB must be 16-byte
 *     aligned (they are read through TMA tensor maps), else MPGEMM_EINVAL.
 * c_ij = RN_DD(2^(e_i + f_j + 2 h) sum_g L_g 2^(-b g)), b = 7, h = 0 (int8)
 * or b = 5, h = 1 (e4m3).  mpgemm_ozaki_split_ex writes 1-byte digits (int8
 * or e4m3 codes) in the layout described for mpgemm_ozaki_split. */
enum { MPGEMM_DIGITS_INT8 = 0, MPGEMM_DIGITS_E4M3 = 1 };
int mpgemm_dd_ozaki_ex(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C,
                       int num_slices, int digit_kind, void* stream);
int mpgemm_ozaki_split_ex(int digit_kind, int by_col, int64_t rows, int64_t cols, const double* X, int num_slices,
                          int* expo, void* digits, void* stream);
int mpgemm_ozaki_levels_ex(int digit_kind, int64_t m, int64_t l, int64_t n, int num_slices, const void* DA,
                           const void* DB, int* levels, void* stream);

/* ---------------------------------------------------------------------------
 * Split-precision QD GEMM (the FP8-digit scheme carried to quad-double; the
 * paper has no counterpart).  A, B, C are QD planes (4 x rows x cols,
 * x_0 leading, canonical: each term at most half an ulp of the one
 * before).  e_i / f_j are the frexp exponents of A's row / B's column
 * maxima of the leading plane; every element is truncated toward zero to
 * 5 S bits of x 2^-(e+1) (exactly, from the exact sum of its four terms),
 * written as S balanced base-32 digits in e4m3, multiplied on the tcgen05
 * tensor cores with exact f32 chunk sums, recombined exactly and rounded
 * greedily to four doubles (x_0 = RN(c), x_1 = RN(c - x_0), ...).
 * num_slices S in 1..48 (0 = 44, which meets 4 l 2^-208 |A||B| on inputs
 * whose entries lie within a few binades of their row / column maxima; see
 * mpgemm_select_precision for the bound).  Limits as for
 * mpgemm_dd_ozaki_ex with e4m3 digits (l <= 65536, S 256 l < 2^31, m and n
 * <= 65535).  Workspace: mpgemm_ozaki_workspace_size(m, l, n, S).
 * mpgemm_ozaki_split_terms: the digit step alone for T-term expansions
 * (terms = 4 only), in the layout of mpgemm_ozaki_split_ex with e4m3
 * digits.
 * ------------------------------------------------------------------------- */
int mpgemm_qd_ozaki(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int num_slices,
                    void* stream);
int mpgemm_qd_ozaki_slices_default(void);
/* The order in which the tcgen05 level kernel (e4m3 digits) runs its jobs,
   one job per 128 x 256 tile of C and level g: tiles grouped into
   super-tiles whose digit planes fit in L2, super-tiles in row-major order,
   within a super-tile the levels from g = S + 1 down to 2.  Host arithmetic
   only: writes (g, first row, first column) of job j to jobs[3j .. 3j + 2]
   for j < max_jobs and returns the number of jobs (tiles x S), or
   MPGEMM_EINVAL for bad sizes (m, n <= 65535). */
int mpgemm_split_job_order(int64_t m, int64_t n, int64_t l, int num_slices, int* jobs, int max_jobs);
int mpgemm_ozaki_split_terms(int terms, int by_col, int64_t rows, int64_t cols, const double* X, int num_slices,
                             int* expo, void* digits, void* stream);

/* ---------------------------------------------------------------------------
 * DD Strassen that allocates nothing.  The paper has no counterpart.  It is
 * for callers that cannot allocate device memory while they run: for
 * example a service whose device memory is all handed to its own pool
 * allocator at start-up, after which nothing else may allocate, or a
 * latency-critical loop that cannot afford an allocation's possible
 * device-wide synchronisation or its failure.  It computes what
 * mpgemm_dd(m, l, n, A, B, C, MPGEMM_STRASSEN, n_min, strassen_depth, stream)
 * computes, with the same kernels, but its workspace is a fixed 32 MiB
 * scratch array inside the library (device memory that every GPU which loads
 * the library holds until the process exits), and it calls no cudaMalloc,
 * cudaFree or other allocating routine.  The caller still passes A, B and C.
 *   - strassen_depth must be 1..4 (MPGEMM_EINVAL otherwise); every other
 *     argument is checked as in mpgemm_dd.
 *   - A problem whose Strassen workspace (mpgemm_workspace_size) is larger
 *     than 32 MiB is refused with MPGEMM_ENOMEM before anything is launched.
 *   - The first call on a device finds the scratch array's device address
 *     (one cudaGetSymbolAddress, made with that device current); make that
 *     first call before any stream capture.
 *   - All calls share the one scratch array.  Calls whose kernels may overlap
 *     on the GPU (different streams with no ordering between them) race on it
 *     and corrupt each other's results: order them on one stream or with
 *     events.  No part of the scratch needs clearing between calls: every
 *     element a call reads was written earlier in the same call.
 * ------------------------------------------------------------------------- */
int mpgemm_dd_strassen_noalloc(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C,
                               int n_min, int strassen_depth, void* stream);

/* ---------------------------------------------------------------------------
 * DD and QD GEMMs on the integer pipe (an extension: the paper computes its
 * DD / QD products with the QD library's floating-point algorithms).  The
 * operands are rounded to p-bit multi-limb numbers, C := AB runs as the
 * multi-limb GEMM (Eqs 1-3, every multiply and add rounded to p bits, as
 * mpgemm_mp), and C is rounded back to 2 (DD) or 4 (QD) doubles.  On GB300
 * the FP64 pipe executes 2 operations per clock per SM, so 128-bit limbs
 * give DD about 1.3x and 256-bit limbs QD about 7.6x the rate of mpgemm_dd
 * / mpgemm_qd (measured at 2048^3 / 1024^3), with a much smaller error (2^-128 / 2^-256 per operation
 * instead of the DD / QD bounds 4 l 2^-104 |A||B| and 4 l 2^-208 |A||B|).
 *   Conversion to p bits (mpgemm_terms_to_mp): c = +0, then for t = 0..T-1
 *     c = RN_p(c + x_t) with the double x_t taken exactly.
 *   Conversion back (mpgemm_mp_to_terms): r = c, then for t = 0..T-1
 *     x_t = RN_53(r) (round to nearest even double) and r = r - x_t (exact):
 *     the greedy expansion of c.
 *   Layouts: A, B, C as for mpgemm_dd (T = 2 planes) or mpgemm_qd (T = 4);
 *   multi-limb planes as for mpgemm_mp.  prec_bits = 32 w, w in {2, 4, 8,
 *   16} (MPGEMM_EUNSUPPORTED otherwise).  algo, n_min, strassen_depth as for
 *   mpgemm_mp at prec_bits (MPGEMM_AUTO uses the multi-limb tuning at
 *   prec_bits).
 *   Workspace: mpgemm_via_mp_workspace_size bytes (the multi-limb copies of
 *   A, B and C plus Strassen's workspace), from mpgemm_set_workspace's
 *   buffer else allocated stream-ordered.
 *   Device status (mpgemm_stream_status): an infinite or NaN input gives
 *   MPGEMM_EINVAL; a result term outside the normal double range is written
 *   as zero and gives MPGEMM_EOVERFLOW.
 * ------------------------------------------------------------------------- */
int mpgemm_dd_via_mp(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int prec_bits,
                     int algo, int n_min, int strassen_depth, void* stream);
int mpgemm_qd_via_mp(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int prec_bits,
                     int algo, int n_min, int strassen_depth, void* stream);
size_t mpgemm_via_mp_workspace_size(int prec_bits, int64_t m, int64_t l, int64_t n, int algo, int strassen_depth);
/* The two conversions alone, over `count` elements: X is terms planes of
   count doubles each (terms = 2 or 4), Y is 2 + prec_bits/32 planes of count
   words.  Device pointers; asynchronous on stream. */
int mpgemm_terms_to_mp(int terms, int64_t count, const double* X, int prec_bits, uint32_t* Y, void* stream);
int mpgemm_mp_to_terms(int terms, int64_t count, int prec_bits, const uint32_t* Y, double* X, void* stream);

/* ---------------------------------------------------------------------------
 * Batched GEMMs of uneven sizes and mixed precisions in one persistent launch
 * (an extension; the paper runs one GEMM at a time).  Each descriptor is one
 * C := AB with its own sizes, format and device pointers (layouts as above).
 *   kind        MPGEMM_KIND_DD, MPGEMM_KIND_QD, or MPGEMM_KIND_MP with
 *               prec_bits = 256 (the only multi-limb width of the batched
 *               kernel)
 *   tile        edge of the C tile one CTA computes: 16 or 32 for DD / QD
 *               (0 = the cost model's choice when one is installed, else
 *               32), always 16 for multi-limb and for engine = 1
 *   engine      0: the format's own arithmetic (FP64 for DD / QD);
 *               1 (DD / QD only, MPGEMM_EINVAL otherwise): the integer
 *               pipe, as mpgemm_dd_via_mp / mpgemm_qd_via_mp with 128 /
 *               256-bit limbs, MPGEMM_BLOCK and n_min = 16.  The plan then
 *               owns multi-limb copies of A, B and C (cudaMalloc at plan
 *               time); each run converts every such A and B in one pass per
 *               format before the persistent kernel and every C in one pass
 *               per format after it (inside the captured graph of
 *               mpgemm_batched_run_graph).
 * mpgemm_batched_plan validates the descriptors (MPGEMM_EINVAL for a
 * negative size, m or n above 65535 * 64, l above 2^31, a NULL matrix of
 * nonzero size, a bad engine or tile; MPGEMM_EUNSUPPORTED for another
 * multi-limb width), builds the table of work
 * items (one per C tile, heaviest first) and copies it to the device
 * (cudaMalloc + synchronous copies: plan outside hot loops).  The plan keeps
 * the pointers; the caller keeps the matrices alive.
 * mpgemm_batched_run resets the plan's work counter and launches the
 * persistent kernel on `stream` (one CTA per resident slot; CTAs take work
 * items from an atomic counter and never wait for each other).  Runs of the
 * same plan must not overlap (they share the counter).
 * mpgemm_batched_run_graph does the same through a CUDA graph captured on the
 * plan's first call (on a stream of the plan's own) and replayed afterwards.
 * mpgemm_batched_sequential runs the same descriptors as one ordinary launch
 * per GEMM (block algorithm, n_min = tile): the baseline.
 * Results are bit-identical to mpgemm_dd / mpgemm_qd / mpgemm_mp with
 * MPGEMM_BLOCK and n_min = tile (engine 1: to mpgemm_dd_via_mp /
 * mpgemm_qd_via_mp as above).
 * ------------------------------------------------------------------------- */
typedef struct {
    int kind;
    int prec_bits;
    int64_t m, l, n;
    const void* A;
    const void* B;
    void* C;
    int tile;
    int engine;
} mpgemm_desc;
typedef struct mpgemm_plan_s* mpgemm_plan;
int mpgemm_batched_plan(const mpgemm_desc* descs, int count, mpgemm_plan* plan);
int mpgemm_batched_run(mpgemm_plan plan, void* stream);
int mpgemm_batched_run_graph(mpgemm_plan plan, void* stream);
int mpgemm_batched_destroy(mpgemm_plan plan);
/* Work items, persistent grid size and the tile chosen for each descriptor. */
int mpgemm_batched_info(mpgemm_plan plan, int* work_items, int* grid, int* tiles, int tiles_len);
int mpgemm_batched_sequential(const mpgemm_desc* descs, int count, void* stream);

/* ---------------------------------------------------------------------------
 * FP32 MLP cost model (an extension standing in for the paper's time
 * prediction, Section 3): log(time) of a configuration (m, l, n, format,
 * precision bits, algorithm, tile, Strassen depth) from 16 features through
 * two hidden layers of 64 ReLU units, trained with Adam by hand-written
 * kernels on timings the library measures itself.  Once trained (or loaded)
 * it is installed for the process: MPGEMM_AUTO then picks, for shapes it has
 * not tuned, among the candidates (simple, block tile 16/32/64, Strassen
 * depth 1..3 with those tiles): when only one is predicted within 30 % of
 * the best (about twice the model's 90th-percentile error) and no other
 * algorithm's best within 60 % or predicted below 2 ms, that one; else
 * those candidates (the ones within 30 % and the best of each algorithm
 * within 60 % or below 2 ms, at most 6) are timed on the call's own
 * operands (10 / 3 / 1 back-to-back runs for predictions below 1 / 20 ms /
 * above; among those within 3 % of the fastest, the fewest launches) and
 * that one is remembered for the shape (and appended to
 * the tuning cache when one is open), so the first such call
 * is synchronous and writes C more than once.  While the stream captures a
 * graph, or in model-only mode (mpgemm_auto_mode(0); 1 restores timing),
 * nothing is timed: among the configurations predicted within 10 % of the
 * best, the one with the fewest launches.  Batched plans use the model for
 * tile = 0.  mpgemm_tune (measured) remains available and wins when it has
 * a remembered choice.
 *   mpgemm_cost_features   feature vector (mpgemm_cost_num_features floats)
 *   mpgemm_cost_collect    time `count` random configurations (shapes
 *                          log-uniform in [16, max_dim], formats DD / QD /
 *                          128- to 1024-bit multi-limb, valid algorithms);
 *                          host output arrays; synchronous; allocates its
 *                          own operand buffers and releases them on every
 *                          path; a failed CUDA call gives MPGEMM_ECUDA, a
 *                          device-side failure of the timed GEMMs their
 *                          stream status
 *   mpgemm_cost_train      train a new model (epochs x count/128 Adam steps,
 *                          lr 2e-3) and install it; optional per-epoch loss
 *   mpgemm_cost_predict    predicted milliseconds for host feature vectors
 *   mpgemm_cost_save/load  binary model file; mpgemm_cost_clear uninstalls
 * ------------------------------------------------------------------------- */
int mpgemm_cost_num_features(void);
/* The installed model's choice for a problem on the stream's SMs (the
   candidate of least predicted time, ignoring remembered tuner choices) and
   its predicted time in ms; MPGEMM_EUNSUPPORTED when no model is installed. */
int mpgemm_cost_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, void* stream, int* algo, int* n_min,
                       int* depth, float* pred_ms);
int mpgemm_cost_features(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int algo, int tile, int depth,
                         float* out);
int mpgemm_cost_collect(int count, unsigned long long seed, int max_dim, float* features, float* times_ms,
                        void* stream);
int mpgemm_cost_train(const float* features, const float* times_ms, int count, int epochs, unsigned long long seed,
                      float* loss_per_epoch);
int mpgemm_cost_predict(const float* features, int count, float* out_ms);
int mpgemm_cost_save(const char* path);
int mpgemm_cost_load(const char* path);
int mpgemm_cost_clear(void);

/* Bytes of workspace one call needs (0 for simple/block). */
size_t mpgemm_workspace_size(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int algo,
                             int strassen_depth);
/* Give the library a device buffer to use as workspace for calls on this
   device (NULL, 0 = allocate per call).  The caller keeps ownership and must
   not free it while calls that may use it are in flight.  Calls on
   different streams that share the buffer must be ordered by the caller. */
int mpgemm_set_workspace(void* dev_ptr, size_t bytes);

/* ---------------------------------------------------------------------------
 * Tuning (Section 3).  mpgemm_tune runs the paper's procedure on the given
 * operands (device pointers in the format of `kind`; C is overwritten):
 *   1. for each n_min in {16, 32, 64, 128, 256, 512} time the block
 *      algorithm on the first r rows of A against all of B, r =
 *      mpgemm_sample_rows(), and predict the full time by scaling T_sample
 *      with the ratio of per-SM rounds of CTAs, ceil(CTAs(m) / SMs) /
 *      ceil(CTAs(r) / SMs) (the paper's m / r when both runs are whole
 *      rounds); SMs = mpgemm_stream_sms(stream);
 *   2. keep the n_min with the smallest prediction;
 *   3. time simple, block(n_min) and Strassen depths 1..3 (leaves at n_min)
 *      and report the fastest.
 * Each timing is the time per run of 3 runs issued back to back after a
 * warm-up run (1 with MPGEMM_TUNE_QUICK): the steady-state cost of a call.
 * With MPGEMM_TUNE_REMEMBER the choice is stored for this (kind, prec_bits,
 * m, l, n, SMs of the stream) and used by MPGEMM_AUTO on streams with as
 * many SMs.  Synchronous; returns MPGEMM_OK or an
 * error status.
 *
 * Persistent tuning cache: mpgemm_tune_cache_open(path) opens (creating it
 * if needed) an append-only file of JSON lines, one record per timing and
 * one per finished choice, keyed by (device name, library version, SMs,
 * kind, prec_bits, m, l, n).  While it is open, mpgemm_tune takes every
 * timing it finds there instead of measuring it and appends (and flushes)
 * every new timing as soon as it is measured, so a run that was killed
 * resumes where it stopped; a shape with a finished choice in the file is
 * answered from it without timing (unless MPGEMM_TUNE_FORCE), and every
 * choice read from the file is remembered for MPGEMM_AUTO, which consults
 * remembered choices before the cost model.  Lines that do not parse are
 * skipped; records of another device name, SM count or version are not
 * used.  Several processes may append to one file.  path NULL closes the
 * cache (remembered choices stay).  MPGEMM_EINVAL if the file cannot be
 * opened or read.  mpgemm_tune_cache_stats: records loaded at open (choices,
 * timings), lines skipped, records of other devices or versions; returns 1
 * while a cache is open, else 0.
 *
 * mpgemm_tune_set_timer(fn, ctx): while fn is not NULL, mpgemm_tune asks fn
 * for each timing (milliseconds; a negative value makes mpgemm_tune return
 * MPGEMM_ECUDA) instead of launching kernels: the procedure can then run on
 * recorded or simulated timings, without a GPU.  NULL restores timing on
 * the device.
 * ------------------------------------------------------------------------- */
enum {
    MPGEMM_TUNE_VERIFY = 1,       /* also time the full block GEMM for every n_min */
    MPGEMM_TUNE_REMEMBER = 2,     /* store the choice for MPGEMM_AUTO               */
    MPGEMM_TUNE_SKIP_SIMPLE = 4,  /* do not time the simple algorithm               */
    MPGEMM_TUNE_QUICK = 8,        /* one timed run per configuration                */
    MPGEMM_TUNE_FORCE = 16        /* tune again although the cache has a choice     */
};
typedef struct {
    int algo, n_min, depth;      /* the choice                                    */
    double best_ms;              /* its measured time                             */
    int n_cand;                  /* candidates below                              */
    int cand_n_min[8];
    int64_t cand_rows[8];        /* rows r of the sample run                      */
    double cand_sample_ms[8];    /* T_sample                                      */
    double cand_pred_ms[8];      /* T_sample * m / r                              */
    double cand_full_ms[8];      /* measured full time (NaN without VERIFY)       */
    double simple_ms, block_ms;  /* NaN when not run                              */
    double strassen_ms[5];       /* [d], d = 1..4; NaN when not run               */
    double tuning_ms;            /* wall time of this call                        */
    int measured;                /* timings taken by this call (not from the cache) */
    int from_cache;              /* 1: the choice came from the tuning cache      */
} mpgemm_tune_report;
int mpgemm_tune(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, const void* A, const void* B, void* C,
                int flags, void* stream, mpgemm_tune_report* report);
/* Forget every remembered choice. */
int mpgemm_tune_forget(void);
int mpgemm_tune_cache_open(const char* path);
int mpgemm_tune_cache_stats(int* choices, int* measurements, int* skipped_lines, int* foreign_records);
typedef double (*mpgemm_timer_fn)(void* ctx, int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int algo,
                                  int n_min, int depth, int64_t rows, int reps);
int mpgemm_tune_set_timer(mpgemm_timer_fn fn, void* ctx);
int mpgemm_auto_mode(int mode);
/* The tuner's timer for one configuration: *ms = the time per call of
   `reps` calls (1..1000) of (algo, n_min, depth) on the operands, issued
   back to back between two events on `stream` after one warm-up call (C is
   overwritten).  Synchronous.  The timer mpgemm_tune and MPGEMM_AUTO use,
   for comparisons on the same footing. */
int mpgemm_time_config(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, const void* A, const void* B,
                       void* C, int algo, int n_min, int depth, int reps, void* stream, double* ms);
/* The (algo, n_min, depth) MPGEMM_AUTO would use for this problem on the
   whole device. */
int mpgemm_auto_choice(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int* algo, int* n_min,
                       int* depth);
/* The paper's prediction (Fig. 1): full time = sampled time * m / rows. */
double mpgemm_predict_time(double t_sample, int64_t m, int64_t rows);
/* Rows r of the sample run for block size n_min: at least 2 n_min (the
   paper's tables give predicted = sampled * m / (2 n_min)), at least one full
   wave of CTAs on `num_sms` SMs, a multiple of the CTA tile, at most m.
   Host arithmetic only. */
int64_t mpgemm_sample_rows(int kind, int64_t m, int64_t n, int n_min, int num_sms);

/* Synchronise `stream`, then read and clear the current device's status
   word: MPGEMM_OK, MPGEMM_EOVERFLOW or MPGEMM_ETIMEOUT. */
int mpgemm_stream_status(void* stream);
/* Self-test of the device failure path (the paper has no counterpart): one
   warp runs the kernels' bounded mbarrier wait on a phase that nothing ever
   completes, with a time limit of limit_ms (1..2000).  The wait gives up,
   the kernel records a timeout in the status word and returns; the call
   synchronises and returns what mpgemm_stream_status reads:
   MPGEMM_ETIMEOUT is the expected result (the status word is cleared and
   the context stays usable).  MPGEMM_EINVAL for a limit out of range. */
int mpgemm_selftest_wait_timeout(int limit_ms, void* stream);
/* Host-side fault injection, for testing callers' error handling (the paper
   has no counterpart).  Arms one fault: the (after + 1)-th device allocation
   (what = MPGEMM_FAULT_ALLOC: Strassen / split-precision / integer-pipe
   workspace, batched plans, precision selection, cost model buffers) or
   launch check (MPGEMM_FAULT_LAUNCH) the library makes from now on fails,
   then the fault disarms; what = MPGEMM_FAULT_NONE disarms.  An injected
   allocation failure allocates nothing and makes the call return
   MPGEMM_ENOMEM (workspace) or the failing API's error; an injected launch
   failure is reported after a launch that did run (MPGEMM_ECUDA,
   mpgemm_last_cuda_error() = 719, a launch failure), so the error paths run
   as for real failures: owned workspace is released on the stream, plans
   are torn down.  Nothing is done to the GPU.  The environment variable
   MPGEMM_FAULT=alloc:N or launch:N arms the same fault at the first call
   that checks it.  mpgemm_fault_fired: faults injected so far. */
enum { MPGEMM_FAULT_NONE = 0, MPGEMM_FAULT_ALLOC = 1, MPGEMM_FAULT_LAUNCH = 2 };
int mpgemm_fault_inject(int what, long long after);
int mpgemm_fault_fired(void);
/* Self-test of the DD / QD kernels' TwoSum: for i < count, out[i] =
   RN(a[i] + b[i]), out[count + i] = its rounding error as the kernels
   compute it (the integer-pipe form) and out[2 count + i] = the same error
   by the FP64 formula y - (s - x).  The two error planes are equal bit for
   bit for every pair of doubles.  Device pointers (out: 3 count doubles);
   asynchronous on stream; MPGEMM_EINVAL for bad arguments. */
int mpgemm_selftest_two_sum(int64_t count, const double* a, const double* b, double* out, void* stream);
/* Self-test of the DD kernel's TwoProd (the product and its rounding error
   on the integer pipe): out[i] = RN(a[i] b[i]) and out[count + i] = its
   error as the kernel computes them, out[2 count + i] = fma(a[i], b[i],
   -p) with p the FP64 product.  out[i] equals the IEEE product (NaN for NaN)
   and the two error planes are equal bit for bit for every pair of doubles.
   Device pointers (out: 3 count doubles); asynchronous on stream;
   MPGEMM_EINVAL for bad arguments. */
int mpgemm_selftest_two_prod(int64_t count, const double* a, const double* b, double* out, void* stream);
/* Self-test of the DD multiply-accumulate step: in = 6 planes of count
   doubles [s, t, ah, al, bh, bl] (accumulator and operands); out = 8 planes:
   [s, t] after the kernels' MAC (TwoProd and TwoSum's error term on the
   integer pipe), [s, t] after the same steps with every error term from
   FP64 operations, then both after one more renormalisation.  The two
   forms are equal bit for bit for every input (NaN as NaN).  Device
   pointers; asynchronous on stream; MPGEMM_EINVAL for bad arguments. */
int mpgemm_selftest_dd_mac(int64_t count, const double* in, double* out, void* stream);
/* Self-test of the DD addition of the Strassen operand and assembly passes
   (Eq 3's sums and differences, each rounded in DD by the accurate
   double-word addition of Joldes, Muller and Popescu 2017): in = 4 planes
   of count doubles [xh, xl, yh, yl]; out = 5 planes: [zh, zl] as the passes
   compute it first (three of its four error terms on the integer pipe),
   [zh, zl] with every error term from FP64 operations, and 1.0 where the
   first form flagged the operands as rare (infinite, NaN or subnormal
   values, or the last Fast2Sum's operands out of exponent order), else
   0.0.  Where the flag is
   0.0 the two results are equal bit for bit; the passes recompute flagged
   elements with the FP64 form.  Device pointers; asynchronous on stream;
   MPGEMM_EINVAL for bad arguments. */
int mpgemm_selftest_dd_add(int64_t count, const double* in, double* out, void* stream);

/* ---------------------------------------------------------------------------
 * Precision selection from an accuracy target (the paper's outlook: choose
 * the precision as well as the algorithm).  Every configuration gets an
 * a-priori elementwise bound |C - AB| <= beta |A||B|:
 *   MPGEMM_SEL_DD           4 l 2^-104 (simple / block);
 *   MPGEMM_SEL_QD           4 l 2^-208 (simple / block);
 *   MPGEMM_SEL_MP           gamma_l = l 2^-p / (1 - l 2^-p), p = prec_bits;
 *   MPGEMM_SEL_OZAKI_INT8 / _E4M3  split precision with S slices: with every
 *       entry at most `spread` binades below the largest of its row of A or
 *       column of B, t = 2^(spread+1-7S) (int8) or 2^(spread+2-5S) (e4m3),
 *       beta = 2t + t^2 + (S+1) c 2^(2 spread + 2 - bS) + 2^-106
 *       (b = 7 / 5, c = 1.02 / 1.07: the truncation of both operands, the
 *       dropped triangle s + t > S + 1, the final DD rounding).
 *   MPGEMM_SEL_DD_VIA_MP / _QD_VIA_MP  DD / QD on the integer pipe with
 *       p-bit limbs (prec_bits; 0 = 128 / 256): gamma_l(p) + 2^(1-p) (the
 *       operands' rounding) + 2^(-53 T) (the final T-term expansion,
 *       T = 2 / 4), with a 2^-40 relative allowance for second-order terms.
 * Strassen is not offered (its bound is normwise, not elementwise).
 *   mpgemm_precision_log2_bound  log2(beta) of one configuration (NaN for
 *                                invalid arguments).
 *   mpgemm_select_precision      the configurations with log2(beta) <=
 *                                log2_target (split precision with the
 *                                fewest slices; the QD split only when
 *                                no DD split meets the target; DD / QD on
 *                                the integer pipe at 128 / 256 bits; the
 *                                smallest multi-limb
 *                                precision of 128..1024 bits), fastest
 *                                first by predicted time (the installed cost
 *                                model's best simple/block configuration,
 *                                else measured GB300 block rates; split
 *                                precision from its tensor work at the
 *                                measured level-kernel rates plus its memory
 *                                passes); writes up to max_out of them to out
 *                                and returns how many there are (>= 0), or
 *                                MPGEMM_EINVAL.  Host only, except that a
 *                                loaded cost model runs its inference kernel.
 * ------------------------------------------------------------------------- */
enum {
    MPGEMM_SEL_DD = 0,
    MPGEMM_SEL_QD = 1,
    MPGEMM_SEL_MP = 2,
    MPGEMM_SEL_OZAKI_INT8 = 3,
    MPGEMM_SEL_OZAKI_E4M3 = 4,
    MPGEMM_SEL_OZAKI_QD = 5,  /* split-precision QD (mpgemm_qd_ozaki), e4m3 digits, final rounding 2^-211 */
    MPGEMM_SEL_DD_VIA_MP = 6, /* mpgemm_dd_via_mp, 128-bit limbs                                           */
    MPGEMM_SEL_QD_VIA_MP = 7  /* mpgemm_qd_via_mp, 256-bit limbs                                           */
};
typedef struct {
    int method;          /* MPGEMM_SEL_*                                  */
    int prec_bits;       /* limb precision (MPGEMM_SEL_MP, _VIA_MP), else 0 */
    int num_slices;      /* split-precision S, else 0                      */
    double log2_bound;   /* log2 of the a-priori bound beta                */
    double est_ms;       /* predicted time                                 */
} mpgemm_precision_choice;
double mpgemm_precision_log2_bound(int method, int prec_bits, int num_slices, int64_t l, int spread);
/* The `spread` of DD operands (A m x l, B l x n, device planes): the largest,
   over rows of A's hi plane and columns of B's hi plane, of (largest frexp
   exponent - smallest frexp exponent of a nonzero entry); 0 for empty or
   all-zero operands.  Using the hi words bounds every |a| from below to
   within a factor 1 - 2^-53.  Synchronous (allocates 4 (2n + 1) bytes
   stream-ordered on `stream`). */
int mpgemm_dd_exponent_spread(int64_t m, int64_t l, int64_t n, const double* A, const double* B, int* spread,
                              void* stream);
int mpgemm_select_precision(double log2_target, int64_t m, int64_t l, int64_t n, int spread,
                            mpgemm_precision_choice* out, int max_out);

/* ---------------------------------------------------------------------------
 * SM partitions (the GPU counterpart of the paper's thread counts, Section
 * 4: every algorithm is timed with 1, 2, 4 and 8 threads).
 *   mpgemm_partition_create   a CUDA green context holding at least num_sms
 *                             SMs (rounded up to the device's partition
 *                             granularity; *sms_out receives the count) and a
 *                             non-blocking stream in it, returned in *stream.
 *                             Every library call issued on that stream runs
 *                             on those SMs only; device memory is shared with
 *                             the rest of the process.  MPGEMM_EUNSUPPORTED
 *                             when the driver has no green contexts,
 *                             MPGEMM_EINVAL for num_sms <= 0 or above the
 *                             device's SM count.
 *   mpgemm_partition_destroy  synchronises the stream, destroys it and its
 *                             green context (MPGEMM_EINVAL for a stream not
 *                             made by mpgemm_partition_create).
 *   mpgemm_stream_sms         SMs the stream's kernels run on: the
 *                             partition's count, else the device's.  The
 *                             tuner's rounds model, remembered choices, the
 *                             cost model's features and the persistent
 *                             tcgen05 kernel's grid use it.
 * A partition only restricts where this process's kernels run; it changes
 * no device setting.  A call on a partition's stream makes the partition's
 * context current on the calling thread for its duration, and a green
 * context can be current on one thread at a time: calls on the same
 * partition must not run concurrently from several host threads.
 * ------------------------------------------------------------------------- */
int mpgemm_partition_create(int num_sms, void** stream, int* sms_out);
int mpgemm_partition_destroy(void* stream);
int mpgemm_stream_sms(void* stream);
const char* mpgemm_strerror(int status);
/* The cudaError_t of the last MPGEMM_ECUDA on this host thread. */
int mpgemm_last_cuda_error(void);
/* Kernel timing for benchmarks: while enabled, every GEMM kernel launch (the
   dominant kernel of each algorithm) is bracketed by CUDA events on its
   stream.  mpgemm_profile_read synchronises on those events and returns the
   summed device milliseconds and the number of launches since the last
   read, then forgets them. */
int mpgemm_profile(int enable);
int mpgemm_profile_read(double* total_ms, int* launches);
/* Library version as 10000*major + 100*minor + patch. */
int mpgemm_version(void);

/* The bounds-checked build of this library (libmpgemm_bc.so, the same
 * sources compiled with -DMPGEMM_BOUNDS_CHECK; a testing tool): every global
 * read and write of the DD / QD / multi-limb simple, block and Strassen
 * kernels (operands, result, each Strassen level's operand and product
 * batches, the integer pipe's limb copies) is checked against the buffer it
 * belongs to.  An access outside is not made (a load reads 0); it is
 * counted and the first such address kept.  mpgemm_bounds_read synchronises
 * the device, returns the count and that address since the last read and
 * clears them.  mpgemm_selftest_bounds launches one thread that reads one
 * element inside a 16-word buffer, one past its end and writes one before
 * its start (the two misses stay inside a larger allocation): a checked
 * build then counts exactly 2.  Both return MPGEMM_EUNSUPPORTED in the
 * normal build.  The counter is per device, not per stream. */
int mpgemm_bounds_read(long long* count, unsigned long long* first_address);
int mpgemm_selftest_bounds(void* stream);

/* ---------------------------------------------------------------------------
 * Peak-rate microbenchmarks (measurement; the paper has no counterpart): the
 * denominators of the rooflines the benchmark reports, measured on the GPU
 * at hand.  mpgemm_peak_run launches `iters` iterations of one instruction
 * loop on every SM of the stream's partition (asynchronous on `stream`) and
 * stores in *ops the operations that launch performs; the caller times the
 * launch with events on the same stream.
 *   MPGEMM_PEAK_TC_E4M3: tcgen05.mma kind::f8f6f4, M 128 x N 256 x K 32,
 *     e4m3 operands resident in shared memory, f32 accumulator in tensor
 *     memory; iters = rounds of 4 MMAs per SM (1..2^22); ops = 2 M N K per
 *     MMA (flops).
 *   MPGEMM_PEAK_MMA_S8: mma.sync m16n8k32 s8 on register operands; ops =
 *     2 x 16 x 8 x 32 per instruction (integer operations).
 *   MPGEMM_PEAK_DFMA: FP64 fused multiply-adds; ops = one per DFMA (the
 *     FP64 operations of the DD / QD rooflines).
 *   MPGEMM_PEAK_IMAD: 32-bit integer multiply-adds; ops = one per IMAD
 *     (thread instructions).
 *   MPGEMM_PEAK_DADD / MPGEMM_PEAK_DMUL: FP64 adds / multiplies; ops = one
 *     per instruction.
 * iters 1..2^32; MPGEMM_EINVAL for a bad kind, count or NULL ops.  The
 * tcgen05 loop's only wait is bounded (a timeout sets the status word). */
enum {
    MPGEMM_PEAK_TC_E4M3 = 0,
    MPGEMM_PEAK_MMA_S8 = 1,
    MPGEMM_PEAK_DFMA = 2,
    MPGEMM_PEAK_IMAD = 3,
    MPGEMM_PEAK_DADD = 4,
    MPGEMM_PEAK_DMUL = 5
};
int mpgemm_peak_run(int kind, int64_t iters, double* ops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPGEMM_H */
