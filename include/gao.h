/*
 * gao.h - C ABI of the GA-driven GPU-offload loop-program library (libgao.so).
 *
 * The method (Yamato et al., "Study of Automatic GPU Offloading Technology for
 * Open IoT", Sec. 3.3 and Sec. 4) takes a program whose parallelisable `for`
 * loops are numbered 0..a-1, encodes an offload pattern as a gene of a bits
 * (bit i = 1: loop i runs on the GPU; 0: it stays on the CPU), measures the
 * program's processing time under that gene, and searches the genes with a
 * Simple GA whose fitness is (processing time)^(-1/2) (Sec. 5.1.2).
 *
 * This library runs such a program on one GPU (sm_103a) and its host CPU:
 *   prog_create  declares the buffers and loops and classifies each loop as
 *                offloadable or not (Sec. 4: the loop list, the parallelisability
 *                check and the gene length a),
 *   prog_run     executes the program under one gene and returns its time
 *                (Sec. 3.3 "evaluation": run the pattern and measure it),
 *   ga_evaluate  scores a population, reusing the time of any gene measured
 *                before (Sec. 4: repeated patterns are not re-measured),
 *   ga_run       runs the whole Simple GA (Sec. 3.3, parameters of Sec. 5.1.2).
 *
 * Conventions for every entry point:
 *   - Return value is a gao_status; GAO_OK = 0.  On error, gao_last_error()
 *     returns a message for the calling thread.  Nothing aborts or traps.
 *   - Arrays passed in are borrowed for the duration of the call only.
 *   - Matrices are row-major binary32; scalars produced by FROBENIUS and SUM
 *     are binary64 (a 1 x 1 buffer of dtype GAO_F64).
 *   - Gene bit k (bit 0 = least significant) places the k-th offloadable loop;
 *     when every loop is offloadable, bit i places loop i.  Bits at or above the
 *     gene length must be zero (GAO_EINVAL otherwise).  At most 64 loops.
 *   - A program is not thread-safe: one call at a time per gao_prog.
 */
#ifndef GAO_H
#define GAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gao_status {
    GAO_OK = 0,
    GAO_EINVAL = 1,   /* invalid argument: null pointer, bad shape, bad gene bits   */
    GAO_ENOMEM = 2,   /* device, pinned-host or arena space exhausted               */
    GAO_ECUDA = 3,    /* a CUDA runtime call failed                                 */
    GAO_ETIMEOUT = 4, /* the run exceeded its time budget (Sec. 5.2: trials time out) */
    GAO_EDEVICE = 5,  /* a kernel raised its error word (bounded wait expired)      */
    GAO_ENODEV = 6,   /* no usable CUDA device of compute capability 10.3           */
    GAO_ECPU = 7      /* a CPU loop failed                                          */
} gao_status;

/* Loop kinds.  The paper's benchmark is a matrix-product program (Sec. 5.1.1)
 * whose loops it does not list; these are the loop bodies the library offers. */
typedef enum gao_loop_kind {
    GAO_LOOP_INIT = 0,      /* outs[t][i,j] = U[-1,1) value of (seed, buffer id outs[t], i*cols+j);
                               flags bit t: multiply row i by its power-of-two factor          */
    GAO_LOOP_GEMM = 1,      /* outs[0] = alpha * ins[0] @ ins[1] + beta * ins[2]; outs[0] may be ins[2] */
    GAO_LOOP_AXPY = 2,      /* outs[0] = ins[0] + alpha * ins[1]   (scale-add D = C + 2A)         */
    GAO_LOOP_TRANSPOSE = 3, /* outs[0] = ins[0]^T                                                */
    GAO_LOOP_ROWSUM = 4,    /* outs[0][i] = sum_j ins[0][i,j]   (rows x 1, binary32)             */
    GAO_LOOP_FROBENIUS = 5, /* outs[0] = sqrt(sum ins[0]^2)     (1 x 1, binary64)                */
    GAO_LOOP_RELU = 6,      /* outs[0] = max(ins[0], 0)                                          */
    GAO_LOOP_SQUARE = 7,    /* outs[0] = ins[0] (.) ins[0]                                       */
    GAO_LOOP_COLMAX = 8,    /* outs[0][j] = max_i ins[0][i,j]   (1 x cols, binary32)             */
    GAO_LOOP_SUM = 9,       /* outs[0] = sum ins[0]             (1 x 1, binary64)                */
    GAO_LOOP_STENCIL3 = 10, /* outs[0][i,j] = sum_{a,b in -1..1} w_ab ins[0][i+a,j+b], ins[0] taken as 0
                               outside the image; the terms with nonzero weight are added in
                               row-major (a, b) order with fused multiply-adds, starting from +0
                               (for finite data the same value as adding all nine).  flags picks
                               w: 0 binomial blur (1 2 1; 2 4 2; 1 2 1)/16, 1 Laplacian
                               (0 1 0; 1 -4 1; 0 1 0), 2 Sobel x (-1 0 1; -2 0 2; -1 0 1),
                               3 Sobel y (-1 -2 -1; 0 0 0; 1 2 1).  The image-analysis loops
                               of the paper's motivating camera workload (Sec. 1).           */
    GAO_LOOP_RECURRENCE = 11, /* outs[0][i,0] = ins[0][i,0];
                               outs[0][i,j] = alpha * outs[0][i,j-1] + ins[0][i,j]  (j >= 1,
                               one fused multiply-add).  Each element depends on the one
                               before it: never offloaded (see gao_offload).                 */
    GAO_LOOP_FIND = 12      /* outs[0][i] = smallest j with ins[0][i,j] > alpha, cols if none
                               (rows x 1, binary64; alpha and the elements compared as
                               binary32).  The loop leaves a row early: never offloaded.     */
} gao_loop_kind;

/* A loop whose body calls an external (host) routine: set this bit in gao_loop.flags.
 * The loop still runs, on the CPU only (see gao_offload). */
#define GAO_LOOP_EXTERNAL_CALL (1ull << 63)

/* Parallelisability of a loop, decided at prog_create.  Sec. 4 tries a parallel
 * directive on each loop and keeps only the loops that compile; the compile errors it
 * names are data dependences between iterations, calls of external routines, loops that
 * exit early (break) and directives at two levels of one nest.  The loops here are whole
 * nests, so the last case cannot occur.  Loops that are not OK run on the CPU under every
 * gene, and the gene has one bit per OK loop (gene length a, Sec. 4). */
typedef enum gao_offload {
    GAO_OFFLOAD_OK = 0,
    GAO_OFFLOAD_DEPENDENCE = 1,    /* loop-carried data dependence (RECURRENCE)        */
    GAO_OFFLOAD_EARLY_EXIT = 2,    /* the loop leaves early (FIND)                     */
    GAO_OFFLOAD_EXTERNAL_CALL = 3  /* flags has GAO_LOOP_EXTERNAL_CALL                 */
} gao_offload;

typedef enum gao_dtype { GAO_F32 = 0, GAO_F64 = 1 } gao_dtype;

typedef enum gao_buf_role {
    GAO_BUF_TEMP = 0,   /* produced and consumed inside the program                               */
    GAO_BUF_INPUT = 1,  /* host data set by prog_set_input; valid on the host at the start of a run */
    GAO_BUF_OUTPUT = 2  /* copied to the host at the end of every run (unless GAO_RUN_KEEP_DEVICE) */
} gao_buf_role;

typedef struct gao_buffer {
    int64_t rows, cols;
    int32_t dtype; /* gao_dtype    */
    int32_t role;  /* gao_buf_role */
} gao_buffer;

#define GAO_MAX_IO 4
typedef struct gao_loop {
    int32_t kind;            /* gao_loop_kind                          */
    int32_t ins[GAO_MAX_IO]; /* buffer indices, -1 for unused slots    */
    int32_t outs[GAO_MAX_IO];
    double alpha, beta;
    uint64_t flags;
} gao_loop;

/* GEMM arithmetic.  Every variant takes binary32 A, B, C and accumulates in binary32. */
typedef enum gao_gemm_prec {
    GAO_GEMM_FP32_SIMT = 0, /* FFMA on the CUDA cores                                      */
    GAO_GEMM_BF16 = 1,      /* A, B rounded to bfloat16, tcgen05 tensor cores              */
    GAO_GEMM_BF16X3 = 2,    /* two-term bfloat16 split, 3 products (hi.hi + hi.lo + lo.hi) */
    GAO_GEMM_BF16X6 = 3,    /* three-term split, 6 products                               */
    GAO_GEMM_FP8 = 4        /* e4m3 with one scale per 128-element K block                */
} gao_gemm_prec;

typedef struct gao_opts {
    int32_t gemm_prec;       /* gao_gemm_prec                                               */
    int32_t kchunk;          /* K elements per binary32 partial sum (0: library default; the
                                FP32 SIMT kernel rounds it up to a multiple of 16)          */
    int32_t tile_cfg;        /* tensor-core tile configuration: bits 0-1 tile width (0 default,
                                1 = 128, 2 = 256 columns; 256 only for plain BF16 without K
                                chunks and for FP8, every other variant uses 128), bit 2 L2
                                prefetch of the operand tiles 4 K blocks ahead (BF16 variants;
                                changes no value), bit 3 CTA pairs: 256-row tiles on two SMs
                                that each load half of every B tile (changes no value),
                                bits 4-7 log2 of the raster group (0: default 16).  The
                                default (0) runs plain BF16 without K chunks and FP8 on
                                256 x 256 pair tiles and the split precisions on 128 x 128
                                tiles of one CTA; prog_autotune picks one                   */
    int32_t cpu_threads;     /* OpenMP threads for CPU loops (0: all)                       */
    uint64_t seed;           /* seed of the INIT loop's counter hash                        */
    double timeout_s;        /* wall-clock budget of one prog_run (0: none)                 */
    void *stream;            /* cudaStream_t the program runs on (NULL: a library stream)   */
    void *dev_arena;         /* caller-owned device memory for every buffer and all scratch
                                (NULL: the library allocates it); must outlive the program */
    uint64_t dev_arena_bytes;
    int32_t transfer_mode;   /* GAO_TRANSFER_RESIDENT or GAO_TRANSFER_PER_LOOP               */
    int32_t fuse_chains;     /* GAO_FUSE_*: whether loop chains that a gene puts on the GPU
                                (resident transfers) run as one pass each:
                                GEMM -> AXPY(C + a X) -> TRANSPOSE [-> ROWSUM] [-> FROBENIUS]
                                of the transpose (tensor-core BF16 precisions: the GEMM's
                                epilogue writes C, D, E, the row sums' block values and the
                                norm's partial sums); linear RELU / SQUARE / AXPY chains;
                                STENCIL3 x2 -> SQUARE x2 -> AXPY [-> SUM] [-> COLMAX] of the
                                magnitude (the gradient chain), with the STENCIL3 that forms
                                its input joining the pass when it is on the GPU too (one pass
                                over the raw image); intermediates no later loop reads are not
                                written.  Results keep the separate loops' bits but for the
                                norm and SUM, which partition their sums differently          */
} gao_opts;

/* Data movement between host and device under a gene (Sec. 2 and Sec. 3.3: CPU-GPU
 * transfers are why naive offloading loses):
 *   RESIDENT  a buffer moves only when a loop needs it on the side where it is not valid;
 *   PER_LOOP  every GPU loop copies its inputs in and its outputs back out, as a directive
 *             offload without a data region does (the paper's measured setting). */
#define GAO_TRANSFER_RESIDENT 0
#define GAO_TRANSFER_PER_LOOP 1

/* Loop-chain fusion: never, whenever the chain is on the GPU, or as the gene decides:
 * GAO_FUSE_GENE adds one bit to the gene, after the loop bits (bit a-1 of a gene of
 * length a), so that the GA chooses fusion like any placement (loop combinations decide
 * the time, Sec. 3.3). */
#define GAO_FUSE_OFF 0
#define GAO_FUSE_ON 1
#define GAO_FUSE_GENE 2

typedef struct gao_prog gao_prog;

/* Device bytes a program needs (buffers + scratch), for callers that supply dev_arena. */
gao_status prog_device_bytes(const gao_loop *loops, int n_loops, const gao_buffer *bufs, int n_bufs,
                             const gao_opts *opts, uint64_t *bytes_out);

/* Declare a program: its buffers and its loops in program order.  Validates shapes and the
 * dataflow (every input is produced earlier or is an INPUT buffer) and classifies every
 * loop (gao_offload); the gene length is the number of offloadable loops.
 * On success *out owns device memory (or uses opts->dev_arena) and pinned host mirrors. */
gao_status prog_create(const gao_loop *loops, int n_loops, const gao_buffer *bufs, int n_bufs,
                       const gao_opts *opts, gao_prog **out);

/* Copy `bytes` of host data into INPUT buffer `buf` (its pinned host mirror). */
gao_status prog_set_input(gao_prog *p, int buf, const void *host_src, uint64_t bytes);

/* Bind caller host memory as buffer `buf`'s host copy (in place of the library's pinned
 * mirror), so that a run copies an INPUT straight from the caller's array to the device
 * and an OUTPUT straight back into the caller's array: no staging copy between the caller's
 * data and the link.  `bytes` must equal the buffer's size.  Memory that is not page-locked
 * already is registered with cudaHostRegister for as long as it stays bound.  An INPUT
 * buffer counts as set from then on; the caller may rewrite the array between runs (the
 * library reads it anew in every run that needs it on the device; the measurement cache
 * is cleared by this call only).  host = NULL unbinds and returns to the library's mirror
 * (an INPUT then needs prog_set_input again).  The memory must stay valid while bound;
 * captured graphs are dropped (they name the old address). */
gao_status prog_bind_host(gao_prog *p, int buf, void *host, uint64_t bytes);

#define GAO_RUN_KEEP_DEVICE 1u /* leave OUTPUT buffers on the device (no final copy) */
#define GAO_RUN_NO_GRAPH 2u    /* plain launches: no CUDA graph is captured or replayed       */
#define GAO_RUN_NO_LOOP_TIMES 4u /* record no per-loop CUDA events (fewer nodes in a captured
                                    graph); prog_stats then reports no loop, copy or kernel
                                    times for the run, the run's own time is unchanged     */

/* Run every loop in program order.  Gene bit k belongs to the k-th offloadable loop in
 * program order (bit i to loop i when every loop is offloadable); that loop runs on the
 * GPU iff the bit is 1, the other loops on the CPU.  Bits at or above the gene length:
 * GAO_EINVAL.  Data moves
 * between host and device only where a loop needs a buffer last written on the other
 * side (Sec. 3.3: CPU-GPU transfers decide which loop combinations are fast).
 * *seconds_out = wall time from the first loop until the outputs are on the host.
 * A gene that puts every loop on the GPU is captured as one CUDA graph the second time it
 * runs (with the same KEEP_DEVICE flag) and replayed from then on: same kernels, copies and
 * per-loop statistics, one launch.  Changing the program's tile configuration
 * (prog_autotune) or prog_cache_clear drops the graphs. */
gao_status prog_run(gao_prog *p, uint64_t gene_mask, uint32_t flags, double *seconds_out);

/* Borrowed pointer to buffer `buf`'s host copy after a run (valid until the next
 * run or destroy); *shape_out receives its shape.  GAO_EINVAL if not on the host. */
gao_status prog_output(gao_prog *p, int buf, const void **host_ptr, gao_buffer *shape_out);

/* Device pointer of buffer `buf` (for callers that keep data on the GPU).  A buffer the
 * last run formed only as a GEMM's bfloat16 planes (prog_planes_for) gets its binary32
 * values formed first (the INIT slot alone, on the program's stream, waited for). */
gao_status prog_device_ptr(gao_prog *p, int buf, void **dev_ptr);

/* INIT into GEMM operand planes: a TEMP buffer that an INIT loop writes and that only one
 * GEMM reads -- as its A or B, on the GPU, in split bfloat16 without a fused chain, with
 * resident transfers -- is formed by the INIT loop straight into that GEMM's bfloat16
 * planes (the counter hash's values split as the GEMM's split kernels would; the GEMM then
 * skips them), and its binary32 array is not written.  *gemm_loop = that GEMM loop if the
 * last run formed buffer `buf` this way and nothing has formed its binary32 values since,
 * else -1.  Anything that reads the buffer afterwards (prog_gemm_residual, prog_device_ptr,
 * prog_autotune) forms it from the INIT slot first. */
gao_status prog_planes_for(const gao_prog *p, int buf, int *gemm_loop);

typedef struct gao_loop_stat {
    int32_t placement;  /* 1: ran on the GPU, 0: on the CPU, 2: on the GPU inside the
                           fused pass of an earlier GEMM loop (its time is that loop's)  */
    int32_t launches;   /* kernels of this library launched for the loop              */
    double device_ms;   /* GPU time of the loop's kernels (CUDA events)                */
    double kernel_ms;   /* GPU time of its main kernel only (GEMM: without the split)  */
    double cpu_ms;      /* host wall time of the CPU loop                              */
    double copy_ms;     /* wall time of the copies issued before the loop              */
    uint64_t h2d_bytes; /* bytes copied host->device before the loop                   */
    uint64_t d2h_bytes; /* bytes copied device->host before the loop                   */
} gao_loop_stat;

/* Gene length a: the number of offloadable loops (Sec. 4), plus one with GAO_FUSE_GENE. */
gao_status prog_gene_length(const gao_prog *p, int *length);

/* Classification of loop `loop`: *verdict = gao_offload, *gene_bit = its bit in the gene,
 * -1 when it is not offloadable.  Either output may be NULL. */
gao_status prog_loop_offload(const gao_prog *p, int loop, int *verdict, int *gene_bit);

/* Per-loop statistics of the last prog_run (n >= loop count). */
gao_status prog_stats(gao_prog *p, gao_loop_stat *out, int n);

/* Number of genes of this program that replay a captured graph, and of genes whose
 * capture failed (they keep running with plain launches).  Either output may be NULL. */
gao_status prog_graphs(const gao_prog *p, int *captured, int *failed);

/* Forget every cached gene time of this program. */
gao_status prog_cache_clear(gao_prog *p);

/* Checkpoint of the search: the program's measured gene times (the cache of Sec. 4), up
 * to cap entries into genes[] and seconds[] (a negative time marks a failed gene);
 * *n_out = the number of entries the cache holds (call with cap = 0 to size the arrays). */
gao_status prog_cache_export(const gao_prog *p, uint64_t *genes, double *seconds, int cap, int *n_out);

/* Resume: put measured times back into the cache (existing entries are kept).  A ga_run
 * with the same parameters and seed then replays the generations already searched without
 * running a program, and measures only genes it has not seen. */
gao_status prog_cache_import(gao_prog *p, const uint64_t *genes, const double *seconds, int n);

void prog_destroy(gao_prog *p);

/* ---- GA (Sec. 3.3 / Sec. 4 / Sec. 5.1.2) ---------------------------------- */

typedef struct gao_ga_params {
    int32_t pop;         /* M, individuals per generation                              */
    int32_t generations; /* T, populations evaluated                                   */
    double pc;           /* crossover rate Pc                                          */
    double pm;           /* mutation rate Pm (per gene)                                */
    int32_t elite;       /* 1: best gene passes unchanged to the next generation       */
    int32_t mutation;    /* 0: flip each gene with prob. pm; 1: flip one gene w.p. pm  */
    uint64_t seed;       /* SplitMix64 seed of all GA draws                            */
    double timeout_s;    /* per-evaluation budget: >0 value, 0 program's own,
                            <0 automatic (10 x the all-GPU time, capped at 60 s)      */
} gao_ga_params;

typedef struct gao_ga_gen {
    uint64_t best_mask; /* best gene of this generation                                 */
    double best_s;      /* its time                                                     */
    double mean_s;      /* mean time over the generation's successful individuals       */
    int32_t evaluated;  /* genes measured for the first time in this generation         */
    int32_t cache_hits; /* individuals whose time came from the cache                   */
    double wall_s;      /* wall-clock seconds of the generation: measuring its new genes
                           and scoring it (host clock)                                  */
} gao_ga_gen;

typedef struct gao_ga_result {
    uint64_t best_mask;   /* best gene found (lowest time; first found on ties)         */
    double best_s;
    int32_t evaluations;  /* distinct genes measured                                    */
    int32_t cache_hits;
    gao_ga_gen *history;  /* optional, caller array of `generations` entries            */
    uint64_t *populations;/* optional, caller array of generations * pop genes          */
} gao_ga_result;

/* Score a population: seconds_out[i] = sum over programs of prog_run time of gene i
 * (from the cache when measured before), fitness_out[i] = seconds^(-1/2), 0 when
 * the gene failed.  *cache_hits_out counts individuals served from the cache. */
gao_status ga_evaluate(gao_prog *const *progs, int n_progs, const uint64_t *population, int pop,
                       double *fitness_out, double *seconds_out, int *cache_hits_out);

/* Run the Simple GA over the programs' common gene length. */
gao_status ga_run(gao_prog *const *progs, int n_progs, const gao_ga_params *params, gao_ga_result *result);

/* Run the same GA against a fixed time table instead of measurements:
 * times[mask] for every mask < 2^n_genes (n_genes <= 24); a negative or
 * non-finite time marks a failed gene (fitness 0).  Host only, no GPU. */
gao_status ga_run_table(const double *times, int n_genes, const gao_ga_params *params, gao_ga_result *result);

/* ---- tile autotuning with the GA ----------------------------------------------- */

/* The Simple GA reused as the tensor-core GEMM's autotuner: a 5-bit gene encodes
 * bits 0-1  raster group of 4, 8, 16 or 32 row tiles per CTA group (L2 reuse order),
 * bits 2-3  split precisions: K chunk of 64, 128, 256 or 512 elements (BF16x6) or 128,
 *           256, 512 or 1024 (BF16x3), all within the stated error bound; plain BF16
 *           and FP8: tile width 128 or 256 columns (bit 2) on one CTA or a CTA pair (bit 3),
 * bit 4     L2 prefetch of the operand tiles (tile_cfg bit 2),
 * and fitness is (measured GEMM time)^(-1/2), the paper's fitness with the kernel time
 * as the benchmark (the GEMM with the loop chain in its epilogue when the program fuses
 * it under the all-GPU gene, since that is the kernel that runs).  The configuration in
 * place is kept unless the GA's best beats it; the result is written into the program's
 * (or the batch's) options and used from then on. */
typedef struct gao_autotune_result {
    int32_t kchunk;     /* best K chunk (0: unchunked)                         */
    int32_t tile_cfg;   /* best tile configuration id (see gao_opts.tile_cfg)  */
    double best_ms;     /* GEMM time of the best configuration                 */
    double default_ms;  /* GEMM time of the configuration in place beforehand  */
    int32_t evaluations;/* configurations measured                             */
    int32_t _pad;
} gao_autotune_result;

/* Tunes the program's GEMM loop (tensor-core precisions); runs the program once under
 * the all-GPU gene first so that the GEMM's inputs are on the device. */
gao_status prog_autotune(gao_prog *p, const gao_ga_params *params, gao_autotune_result *out);

/* ---- batched evaluation over a program suite ---------------------------------- */

/* A batch scores genes over a suite of programs that share one loop structure (same
 * loop kinds in the same order, same GEMM precision), e.g. six-loop programs of many
 * sizes.  A gene runs on every program at once, loop by loop: on the GPU all programs'
 * loop i is one CUDA graph launch (captured by batch_create; small kernels of different
 * programs run concurrently), a tensor-core GEMM loop is the captured operand splits plus
 * ONE grouped persistent tcgen05 launch over every program's tiles, and on the host the
 * programs' loops run one after another.  The gene's time is the wall time of the whole
 * suite, boundary copies included; a gene measured before is served from the batch's
 * cache (Sec. 4).  The programs stay owned by the caller, must outlive the batch, and must
 * not run elsewhere meanwhile; each program's host and device buffers hold its results
 * after a gene runs.  All programs share one fuse_chains setting (GAO_FUSE_OFF or
 * GAO_FUSE_ON; GAO_FUSE_GENE is refused: batch genes are loop placements only).  With
 * GAO_FUSE_ON a gene that puts a program's GEMM -> scale-add -> transpose [-> row sums]
 * [-> norm] chain on the GPU runs the chain in the grouped launch's epilogue,
 * bit-identical to the separate loops but the norm (within its reduction's rounding).
 * The INIT loop (without row scaling) of all programs is one grouped launch too.
 *
 * Generations (batch_set_replicas with R > 1): the batch makes R - 1 copies of the suite
 * (same loops, buffers, options and INPUT data; library-owned device memory), and the
 * new genes of a population or GA generation are measured up to R at a time: gene r runs
 * on copy r, the copies' phases go one after another on the batch's stream, and the
 * GEMMs of every one of these genes that offloads the GEMM loop -- genes x programs --
 * run in ONE grouped persistent launch.  Since genes share that launch, a gene's time is
 * attributed: the device time of its own phase graphs and boundary copies (CUDA events
 * around each), the span of its own problems inside the grouped launch (global-timer
 * stamps taken by the kernel when it starts a tile's loads and when it has stored a tile),
 * and the host wall time of its CPU loops.  That omits the host's launch overheads, so it
 * reads a little below the gene's wall time when run alone; gene rankings carry over
 * (measured, see the tests and the bench).  With a budget, a gene whose attributed time
 * passes it is cut off at the budget.  Results land in the copy that ran the gene; the
 * caller's programs hold the results of the first gene of the last group. */
typedef struct gao_batch gao_batch;

typedef struct gao_batch_stat {
    int64_t executed;          /* genes measured                                        */
    int64_t served;            /* genes answered from the cache                         */
    double exec_seconds;       /* host wall time spent measuring genes                  */
    double gemm_phase_ms;      /* GPU time of the last grouped GEMM launch (events around
                                  it; the operand splits are part of the GEMM loop's
                                  phase graph before it)                                 */
    double gemm_flops;         /* 2MNK summed over that launch's GEMMs (over the suite
                                  before any launch)                                     */
    int32_t gemm_tiles;        /* CTAs (output tiles) of that launch                    */
    int32_t launches_per_gene; /* kernels the all-GPU gene launches                     */
    int32_t graphs;            /* phase graphs captured for the suite                   */
    int32_t fused_phases;      /* GEMM phases run with the loop chain in the epilogue
                                  (programs created with GAO_FUSE_ON; genes measured)     */
    int64_t kernel_launches;   /* kernels launched by the genes measured so far (the
                                  kernels of every phase graph and grouped launch)       */
    int64_t grouped_launches;  /* grouped GEMM launches made by measured genes          */
    int64_t grouped_genes;     /* genes those launches served, summed: with generations
                                  several genes share one launch                         */
    int32_t replicas;          /* copies of the suite (genes measured together)         */
    int32_t _pad;
} gao_batch_stat;

gao_status batch_create(gao_prog *const *progs, int n_progs, gao_batch **out);
/* Measure up to `replicas` genes together (1: one gene at a time, wall-time measurement;
 * > 1: generations share one grouped GEMM launch, attributed times, see above).  Makes or
 * frees copies of the suite and clears the batch's cache.  At most 256. */
gao_status batch_set_replicas(gao_batch *b, int replicas);
/* Program `index` of copy `replica` of the suite (copy 0: the caller's own programs), a
 * borrowed pointer valid until the copy is freed (batch_set_replicas, batch_destroy): the
 * copy that ran a gene holds that gene's results (prog_output, prog_device_ptr). */
gao_status batch_replica_prog(gao_batch *b, int replica, int index, gao_prog **out);
/* Same contract as ga_evaluate, for genes over the whole suite. */
gao_status batch_evaluate(gao_batch *b, const uint64_t *population, int pop, double *fitness_out,
                          double *seconds_out, int *cache_hits_out);
/* The Simple GA with batched evaluation (same draws as ga_run); each generation's new
 * genes are measured together when the batch has replicas. */
gao_status batch_ga_run(gao_batch *b, const gao_ga_params *params, gao_ga_result *result);
gao_status batch_stats(gao_batch *b, gao_batch_stat *out);
/* Tunes the batch's grouped GEMM launch (same gene as prog_autotune; the time is the
 * GEMM loop's splits and grouped launch over the suite), for every copy of the suite. */
gao_status batch_autotune(gao_batch *b, const gao_ga_params *params, gao_autotune_result *out);
void batch_destroy(gao_batch *b);

/* Measures n genes (distinct, not measured before); writes seconds_out[i] (negative or
 * non-finite for a failed gene) and returns GAO_OK, or another status to stop the GA. */
typedef int (*gao_gene_eval_fn)(const uint64_t *genes, int n, double *seconds_out, void *ctx);

/* The Simple GA with a caller-supplied evaluation of each generation's new genes (same
 * draws as ga_run).  Lets a caller measure a generation's genes in parallel, e.g. one
 * process per GPU, each measuring a share and exchanging the times. */
gao_status ga_run_callback(int n_genes, const gao_ga_params *params, gao_gene_eval_fn eval, void *ctx,
                           gao_ga_result *result);

/* ---- residual check of a GEMM on the GPU, in binary64 ------------------------ */

/* Freivalds' check (Freivalds 1977) of C = alpha A B + beta C0, the GEMM loop of the
 * paper's matrix-product benchmark (Sec. 5.1.1), without forming the product again: for
 * vectors x (N entries) and y (M entries) the identities
 *     C x   = alpha A (B x)   + beta C0 x          (right form)
 *     y^T C = alpha (y^T A) B + beta y^T C0        (left form)
 * hold exactly for the exact product, and every entry of C enters both.  With the
 * residual vectors r = C x - beta C0 x - alpha A (B x) (M entries) and s = y^T C -
 * beta y^T C0 - alpha (y^T A) B (N entries) and the reference sides f = alpha A (B x)
 * + beta C0 x and g = alpha (y^T A) B + beta y^T C0:
 *     right = ||r||_2 / ||f||_2,   right_inf = max|r_i| / max|f_i|,
 *     left  = ||s||_2 / ||g||_2,   left_inf  = max|s_j| / max|g_j|,
 * and right_argmax / left_argmax the first i (j) where |r_i| (|s_j|) is largest: a single
 * wrong entry C_ij + d moves r_i by d x_j and s_j by d y_i and nothing else.  Every product
 * and sum runs in binary64 on the GPU (the binary32 inputs are exact in binary64), in a
 * fixed order (the same inputs give the same bits).  Random sign vectors x, y make the
 * check miss an error only with probability <= 1/2 per form (Freivalds 1977). */
typedef struct gao_residual {
    double right, left;
    double right_inf, left_inf;
    int64_t right_argmax, left_argmax;
} gao_residual;

/* Device scratch bytes gao_gemm_residual needs for an M x N x K GEMM (M, N >= 1, K >= 0). */
gao_status gao_gemm_residual_scratch(int64_t M, int64_t N, int64_t K, uint64_t *bytes);

/* The check on caller-owned device data: A (M x K), B (K x N), C0 and C (M x N), row-major
 * binary32; C0 may be NULL (beta term absent); x (N) and y (M) binary64 device vectors;
 * scratch: device memory of at least gao_gemm_residual_scratch bytes, 256-byte aligned.
 * r_out (M doubles) and s_out (N doubles) receive the residual vectors when not NULL
 * (device memory).  Runs on `stream` (NULL: the legacy default stream) and waits for it;
 * *out is filled on return.  Allocates nothing. */
gao_status gao_gemm_residual(const float *A, const float *B, const float *C0, const float *C, int64_t M, int64_t N,
                             int64_t K, double alpha, double beta, const double *x, const double *y, void *scratch,
                             uint64_t scratch_bytes, double *r_out, double *s_out, gao_residual *out, void *stream);

/* The same check of GEMM loop `loop` of a program after a run, on the program's own device
 * buffers and scratch: x (N doubles) and y (M doubles) are host arrays.  The loop's C0
 * must be a buffer of its own (a GEMM that writes C over C0 leaves nothing to check
 * against: GAO_EINVAL); a buffer valid only on the host is copied to the device first. */
gao_status prog_gemm_residual(gao_prog *p, int loop, const double *x, const double *y, gao_residual *out);

/* ---- misc ------------------------------------------------------------------ */

/* Message of the last failing call on this thread ("" if none). */
const char *gao_last_error(void);

/* Library version string. */
const char *gao_version(void);

/* Device-side wait self-test: launches one kernel that waits for a flag nothing
 * sets, with a wall-clock limit of limit_s; the kernel records the expiry in the
 * library's error word and returns.  Returns GAO_ETIMEOUT when the limit was
 * observed (the expected outcome), GAO_OK never.  stream may be NULL. */
gao_status gao_selftest_device_wait(double limit_s, void *stream);

/* ---- allocation-free variant ------------------------------------------------ */

/* Column maxima out[j] = max_i in[i][j] of a rows x cols row-major binary32 matrix
 * already on the device, written to dev_out (cols binary32 values, device memory);
 * the same result as a GAO_LOOP_COLMAX loop.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they need
 * the result -- code running under a host framework whose pool allocator owns the
 * GPU's memory, or a latency-critical loop that cannot afford cudaMalloc/cudaFree
 * (which may synchronise the device and can fail with out-of-memory mid-run).
 *
 * It allocates nothing and calls no allocating routine.  Its scratch, one 32-bit key
 * per column, is a fixed array of GAO_COLMAX_NOALLOC_MAX_COLS keys (256 KiB) inside
 * the library; every GPU that loads the library holds that array until the process
 * exits.  cols above the maximum is rejected with GAO_EINVAL.  The first call on a
 * device (with that device current) looks up the array's device address; make that
 * first call before any stream capture.  Every call clears the keys it uses on
 * `stream` before reducing, and all calls share the one array: calls whose work
 * overlaps on the GPU (different streams, or several host threads) race and give
 * wrong results.  Asynchronous on `stream` (NULL: the legacy default stream);
 * dev_in and dev_out are owned by the caller. */
#define GAO_COLMAX_NOALLOC_MAX_COLS 65536
gao_status gao_colmax_noalloc(const float *dev_in, int64_t rows, int64_t cols, float *dev_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GAO_H */
