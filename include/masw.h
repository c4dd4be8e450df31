/*
 * masw.h -- C ABI of libmasw, a GB300-native engine for theoretical
 * Rayleigh-wave dispersion curves (the forward problem of MASW inversion,
 * Kump & Martin, "MASWAccelerated").
 *
 * Problem statement (Section 2.1, Algorithm 1): a model M has N finite layers
 * (thickness h, P speed alpha, S speed beta, density rho) over a half-space.
 * For each wavelength lambda in W and test velocities V[0] < V[1] < ..., the
 * theoretical velocity C_t(lambda) is the first V[n] whose stiffness-matrix
 * determinant det K(k = 2 pi / lambda, c = V[n]) differs in sign from that of
 * V[n-1]. K is the 2(N+1) x 2(N+1) banded stiffness matrix of the stiffness
 * matrix method. The misfit (Algorithm 2) compares C_t with an observed curve
 * C_e.
 *
 * Conventions shared by every call:
 *  - Units: metres, metres per second, kilograms per cubic metre.
 *  - Ragged batches: models are concatenated. Model m has n_layers[m] = N_m
 *    finite layers; h holds N_m values, alpha/beta/rho hold N_m + 1 (the last
 *    is the half-space); lambda holds n_lambda[m] values. An "item" is one
 *    (model, wavelength) pair; item order is the concatenated lambda order.
 *  - Grid: V[n] = c0 + n * dc, rounded once (fused multiply-add), n < n_c.
 *    Only V[n] < beta of the half-space is scanned (the half-space stiffness
 *    is complex above it). No sign change there -> per-item status
 *    MASW_NO_ROOT, C_t = NaN, index -1.
 *  - sgn(x) = (x > 0) - (x < 0); an exact zero determinant counts as a change.
 *  - C_t is the upper end V[n] of the first sign-changing pair.
 *  - Every call enqueues its GPU work on the batch's stream. Calls that write
 *    host memory synchronise that stream before returning; calls that only
 *    write device memory return without synchronising.
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; all buffers are owned by the caller and are
 *    only read or written during the call (or, for device outputs, by work
 *    the call enqueued).
 *  - Return value: MASW_OK (0) or a positive MASW_E* code; masw_strerror
 *    gives its text. On a validation error no output is written.
 */
#ifndef MASW_H
#define MASW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- call status codes ---- */
#define MASW_OK 0
#define MASW_EINVAL 1   /* invalid argument or model (h<=0, rho<=0, beta<=0, alpha^2 <= 4/3 beta^2, NaN, ...) */
#define MASW_ENOMEM 2   /* device or host allocation failed */
#define MASW_EADMIT 3   /* serving: request refused by the slot or memory cap */
#define MASW_ECUDA 4    /* a CUDA runtime call failed */
#define MASW_ETIMEOUT 5 /* serving: a bounded wait ran out */
#define MASW_EAGAIN 6   /* serving: result not ready yet */
#define MASW_ETOOBIG 7  /* batch exceeds the fixed scratch of masw_dispersion_noalloc */

/* ---- per-item status ---- */
#define MASW_FOUND 0
#define MASW_NO_ROOT 1

/* ---- memory spaces ---- */
#define MASW_HOST 0
#define MASW_DEVICE 1

/* ---- misfit kinds ---- */
#define MASW_MISFIT_PAPER 0 /* Algorithm 2: (1/L) sum |C - C_e| / C_e */
#define MASW_MISFIT_LSQ 1   /* 1/(2 sigma^2) sum (C - C_e)^2 */

/* Library limits. */
#define MASW_MAX_LAYERS 128 /* finite layers per model */

typedef struct masw_batch masw_batch;

/* Ragged model batch (Section 2.1, "model parameter inputs M" and "W").
 * mem_space tells where ALL pointers of this struct live. */
typedef struct {
    int32_t n_models;
    const int32_t* n_layers; /* [n_models] N_m >= 0 */
    const double* h;         /* [sum N_m]           thickness, > 0 */
    const double* alpha;     /* [sum N_m + 1]       P speed, alpha^2 > 4/3 beta^2 */
    const double* beta;      /* [sum N_m + 1]       S speed, > 0 */
    const double* rho;       /* [sum N_m + 1]       density, > 0 */
    const int32_t* n_lambda; /* [n_models] >= 0 */
    const double* lambda;    /* [sum n_lambda]      wavelength, > 0 */
    int32_t mem_space;       /* MASW_HOST or MASW_DEVICE */
} masw_models_desc;

/* Test velocities V (Algorithm 1): V[n] = c0 + n*dc, c0 > 0, dc > 0, n_c >= 2. */
typedef struct {
    double c0;
    double dc;
    int32_t n_c;
} masw_grid;

/* Launch plan of the scan (see masw_autotune). */
typedef struct {
    int32_t warps_per_block; /* 1, 2, 4, 8 */
    int32_t cpl;             /* test velocities per lane per chunk: 1, 2, 4 (precision 1 with
                                2: two adjacent points per lane in packed FP32x2 arithmetic) */
    int32_t blocks_per_sm;   /* persistent grid = blocks_per_sm x SM count */
    int32_t persistent;      /* 1: warps pop items from a work queue */
    int32_t ordered;         /* 1: queue ordered by predicted scan length (longest first) */
    int32_t stage_layers;    /* layer records staged in shared memory per warp (0: none) */
    int32_t use_graph;       /* 1: replay the scan as a captured CUDA graph */
    int32_t precision;       /* 0: FP64 scan of every test velocity; 1: FP32 screen locates the
                                first change, FP64 decides it (V[0], V[n-1], V[n], then an FP64
                                window or full re-scan when they disagree); 2: as 1, but the
                                FP32 change is located by a Wittrick-Williams counting search
                                (bisection on the number of negative eigenvalues of K below
                                the pole-free bound min_i beta_i sqrt(1 + (pi/(k h_i))^2)),
                                certified in FP64 by count 0 at V[n-1] and odd at V[n]; items
                                outside the bound take the linear screen of 1. Default: 2 */
    int32_t count_block;     /* precision 2: threads per block of the counting kernel, 64, 128
                                or 256 (two lanes per item, items of a block consecutive;
                                launch bounds of 14, 7 or 2 resident blocks). Default: 256
                                with count_split 2, else 128 */
    int32_t count_split;     /* precision 2: 0 the search (a lane pair per item, three-way
                                splits) and the certificate in one kernel; 1 the search
                                in kernels of their own (one thread per item: every 6th
                                wavelength of a model and its last by bisection, then
                                the others from a guess between those two indices)
                                before the certificate's; 2 as 1, and the items the
                                search passes straight to the linear FP32 scan (no count
                                change below the bound, a mode below V[0]) take that
                                scan, its check and the mode-count search on a second,
                                highest-priority stream beside the certificate. Same
                                results for all three. Default by batch size: 0 below
                                131,072 items, 1 below 262,144, else 2. With 1 or 2,
                                count_block 64 gives the certificate kernel 640 resident
                                threads (96 registers) */
} masw_plan;

/* Copy and validate a model batch into batch-owned device memory and bind it
 * to cuda_stream (a cudaStream_t; NULL = legacy default stream). The caller
 * keeps ownership of every input pointer; they are read during the call only.
 * Errors: MASW_EINVAL (any invalid value, n_models < 1, N_m > MASW_MAX_LAYERS),
 * MASW_ENOMEM, MASW_ECUDA. *out is set only on success. */
int masw_model_batch_create(const masw_models_desc* models, const masw_grid* grid,
                            void* cuda_stream, masw_batch** out);

/* Release the batch and everything it owns (waits for its stream). */
int masw_model_batch_destroy(masw_batch* batch);

/* Replace the layer parameters of an existing batch (same n_layers and
 * n_lambda; wavelengths unchanged). Pointers live in mem_space. The layer
 * records and the scan limits are rebuilt on the GPU, queued after the work
 * already on the batch stream. MASW_HOST: the arrays are checked on the host
 * with the rules of masw_model_batch_create (MASW_EINVAL before anything is
 * queued) and the call returns without synchronising; the copies read the
 * arrays when the stream reaches them, so pinned (page-locked) arrays must
 * stay unchanged until the batch stream next synchronises (any call with host
 * outputs does), while pageable ones are staged before the call returns.
 * MASW_DEVICE: the checks run on the GPU and the call synchronises the stream
 * once to return their result. MASW_EINVAL leaves the batch unchanged.
 * Used by inversion loops and samplers; a captured scan graph stays valid. */
int masw_model_batch_update(masw_batch* batch, const double* h, const double* alpha,
                            const double* beta, const double* rho, int32_t mem_space);

/* Set beta_i (sum(N_m + 1) values) and h_i (sum(N_m)) of every layer with
 * each layer's Poisson ratio and density held, i.e. alpha_i = beta_i *
 * (alpha_i/beta_i as created): the parameters of masw_misfit_grad. Runs on
 * the GPU (host or device pointers); synchronises the batch stream to
 * report MASW_EINVAL for a non-positive or non-finite value. Used by
 * gradient-based inversion loops; the processing order is kept. */
int masw_model_batch_update_beta_h(masw_batch* batch, const double* h, const double* beta);

/* Number of items (sum of n_lambda) and models of the batch. */
int masw_batch_info(const masw_batch* batch, int64_t* n_items, int32_t* n_models,
                    int32_t* max_layers);

/* Algorithm 1 for every item. Outputs (length n_items, item order) live in
 * out_mem_space: ct = C_t (NaN when not found), ct_idx = n (-1 when not
 * found), status = MASW_FOUND / MASW_NO_ROOT. Any output pointer may be NULL.
 * Uses the batch plan (persistent, ordered, graph-replayed by default). */
int masw_dispersion(masw_batch* batch, double* ct, int32_t* ct_idx, int32_t* status,
                    int32_t out_mem_space);

/* The plain comparison path: one scan launch per model (one curve per
 * launch), synchronising the stream after each model -- the paper's
 * one-curve-per-call GPU pattern (Section 2.3). Same outputs as
 * masw_dispersion. */
int masw_dispersion_plain(masw_batch* batch, double* ct, int32_t* ct_idx, int32_t* status,
                          int32_t out_mem_space);

/* Algorithm 2 per model after running Algorithm 1: ce (host or device,
 * length n_items, item order) is the observed curve C_e; misfit (host or
 * device, length n_models). kind = MASW_MISFIT_PAPER or MASW_MISFIT_LSQ
 * (sigma > 0 used by LSQ only). A model with an item without root gets NaN. */
int masw_misfit(masw_batch* batch, const double* ce, int32_t kind, double sigma, double* misfit);

/* One whole evaluation with every result returned: Algorithm 1 for every item
 * and Algorithm 2 per model, then C_t and the misfit copied out together, as
 * the paper's GPU procedure copies both back to the host at its end (Section
 * 2.3). ce and misfit as masw_misfit; ct, ct_idx, status as masw_dispersion
 * (any may be NULL). Each pointer may be host or device memory on its own.
 * Host buffers are read and written by asynchronous copies on the batch
 * stream, and the call synchronises that stream once, at its end, when any
 * of them is host memory (pinned host memory makes the copies fastest);
 * with device pointers only it returns without waiting. */
int masw_misfit_curves(masw_batch* batch, const double* ce, int32_t kind, double sigma,
                       double* misfit, double* ct, int32_t* ct_idx, int32_t* status);

/* Misfit evaluated on the refined continuous roots C* (bisection inside the
 * first sign-changing bracket to a relative width of 1e-13) and its exact
 * gradient by the implicit-function rule d(C*)/d(theta) = -(u^T dK/dtheta u) /
 * (u^T dK/dc u), u the null vector of K(C*). theta = beta_i (Poisson ratio
 * held: alpha_i moves with beta_i) and h_i. grad_beta has sum(N_m + 1)
 * entries, grad_h sum(N_m), both concatenated like beta and h. All outputs
 * host or device; any may be NULL except misfit. */
int masw_misfit_grad(masw_batch* batch, const double* ce, int32_t kind, double sigma,
                     double* misfit, double* grad_beta, double* grad_h);

/* Wittrick-Williams counts of K(k_item, c) at n arbitrary points, by the
 * arithmetic of the mode-count search: s = the number of negative eigenvalues
 * of K (Sylvester's inertia of the 2x2 Schur pivots), j0 = the number of
 * modes below c of the finite layers with both faces clamped (each layer's
 * thickness halved until c lies under the pole-free bound). s + j0 is the
 * number of modes of the layered structure below c. item, c, s, j0: host or
 * device, length n. Points with c outside (0, beta_halfspace), or whose
 * rescaling failed, get -1 in both. */
int masw_mode_count(masw_batch* batch, int32_t n, const int32_t* item, const double* c,
                    int32_t* s, int32_t* j0);

/* Refined roots C* per item (host or device, length n_items; NaN where
 * Algorithm 1 found none). */
int masw_roots(masw_batch* batch, double* croot);

/* d(C*)/d(theta) per item: rows of 2 N_m + 1 values (dbeta_0..dbeta_N,
 * dh_0..dh_{N-1}) concatenated in item order (host or device). *row_len_total
 * receives the total length when rows is NULL. */
int masw_root_grad(masw_batch* batch, double* rows, int64_t* row_len_total);

/* Sign and ln|det K(k_item, c)| at n arbitrary points (parity checks of the
 * block recurrence). item, c, sign, log_abs: host or device, length n.
 * Points with c outside (0, beta_halfspace) get sign 0 and NaN. */
int masw_det_eval(masw_batch* batch, int32_t n, const int32_t* item, const double* c,
                  int32_t* sign, double* log_abs);

/* Current plan of the batch; set a plan (validated; the graph is rebuilt). */
int masw_get_plan(const masw_batch* batch, masw_plan* plan);
int masw_set_plan(masw_batch* batch, const masw_plan* plan);

/* Time candidate plans on this batch (median of reps timed scans each,
 * CUDA events on the batch stream), keep the fastest, return it in *best
 * (may be NULL). The search is staged: the counting kernel's block size and
 * count_split (precision 2), then warps_per_block x blocks_per_sm, then cpl x ordered,
 * each stage keeping the best of the previous ones, and last the flat
 * (non-persistent) launch. Results never depend on the plan. Winners are cached per (max layers,
 * n_c, item-count bucket) in-process and, when the environment variable
 * MASW_PLAN_CACHE names a file, across processes. */
int masw_autotune(masw_batch* batch, int32_t reps, masw_plan* best);

/* Device time (ms) of the most recent scan launched by masw_dispersion or
 * masw_dispersion_plain (CUDA events on the batch stream). */
int masw_last_scan_ms(const masw_batch* batch, float* ms);

/* Device time (ms) of the three phases of the most recent two-precision
 * scan launched without a graph (plan use_graph 0), from CUDA events between
 * the launches on the batch stream. Plan precision 1: ms[0] FP32 screen,
 * ms[1] FP64 check, ms[2] FP64 re-scan. Plan precision 2: ms[0] counting
 * search with its FP64 certificate (see masw_last_count_phases), ms[1] linear FP32 scan
 * and FP64 check of the fallback items and the FP64 mode-count search of the
 * items that failed a check, ms[2] FP64 re-scan (items whose FP64 counts
 * failed). Plan precision 1: ms[1] also includes that search. MASW_EINVAL when that
 * scan was graph-replayed. */
int masw_last_scan_phases(const masw_batch* batch, float* ms);

/* Three device times (ms) of the most recent scan launched without a graph,
 * for a plan with precision 2 and count_split 1 or 2: ms[0] the FP32
 * counting search (count_search_kernel), ms[1] its FP64 certificate
 * (count_certify_kernel), ms[2] with count_split 2 the fallback chain on the
 * second stream, from the end of the search to its last kernel (it runs
 * beside the certificate), else 0. ms[0] + ms[1] is the first phase of
 * masw_last_scan_phases. MASW_EINVAL for other plans and for a graph-replayed
 * or per-model (masw_dispersion_plain) scan. */
int masw_last_count_phases(const masw_batch* batch, float* ms);

/* The FP32 screen's first-change index per item (item order, -1 when the
 * screen saw none) from the most recent two-precision scan, host or device
 * buffer of n_items; a diagnostic of how well the screen locates roots.
 * Under plan precision 2, bit 30 (MASW_SCREEN_COUNTED) is set on items whose
 * index the counting search located and the FP64 count certified. */
#define MASW_SCREEN_COUNTED (1 << 30)
int masw_last_scan_screen(masw_batch* batch, int32_t* n32);

/* Test hook: the k-th next device allocation made by the library's batch
 * entry points fails with MASW_ENOMEM (k = 0: the next one; once), so that
 * tests can check that every partial failure is reported and cleaned up;
 * k < 0 disables it. Process-wide and not synchronised with other threads:
 * for tests only. */
int masw_test_fail_alloc(int32_t k);

/* Test routing of the two-precision and counting plans, so that tests can
 * run every item through the paths that ordinary inputs rarely reach; the
 * results must not change. 0: normal. 1: the counting search's items all go to
 * the linear FP32 scan from V[0] (plan precision 2). 2: also, every item fails
 * its three-point FP64 check and takes the FP64 mode-count search. 3: also,
 * every searched item takes the FP64 scan from V[0], every higher-mode item
 * the FP64 scan at every grid point, and every item of the leaky
 * continuation the FP64 scan after its double-float one. 4 (no other routing): each
 * higher-mode event that the FP32 search locates is displaced by 0, -1, +1,
 * +3 or -7 grid points (by item index mod 5) before its FP64 certificate, so
 * that the search's recovery steps run. Synchronises the batch stream and
 * rebuilds the scan graph. MASW_EINVAL outside 0..4. */
int masw_set_route(masw_batch* batch, int32_t route);

/* Items of the most recent two-precision scan (plan precision 1 or 2) whose FP32
 * result failed its FP64 check (the counting certificate, or the three-point
 * check on the Wittrick-Williams mode count) and whose first change was then
 * searched on the FP64 mode count from V[0] (-1 for a precision-0 plan).
 * Synchronises the batch stream. */
int masw_last_scan_unresolved(const masw_batch* batch, int32_t* n);

/* ---------------------------------------------------------------------
 * Higher modes. The paper keeps only the first sign change (Algorithm 1,
 * Section 2.1) and names no higher modes; this carries the same scan past it.
 * --------------------------------------------------------------------- */
#define MASW_MAX_CHANGES 15

/* The first max_changes (1..MASW_MAX_CHANGES) sign changes of det K(k, V[n])
 * along the grid for every item: the n >= 1, in increasing order below the
 * scan limit (V[n] < beta_halfspace), whose sign differs from V[n-1]'s
 * (Algorithm 1 stops at the first). Each change carries delta_count, the
 * change in the number of negative eigenvalues of K across it
 * (Wittrick-Williams): +1 where a mode of the layered structure is crossed
 * (a root of det K: the fundamental, then higher modes), -1 at a pole (a
 * mode of one layer with both faces clamped, where det K changes sign
 * through infinity), other values where both fall between two grid points.
 * Outputs are [n_items][max_changes] in item order (host or device buffers
 * per out_mem_space, any may be NULL): ct = V[n] (NaN when fewer changes),
 * ct_idx = n (-1), status MASW_FOUND / MASW_NO_ROOT, delta_count (0). The
 * first change is masw_dispersion's (the batch plan). Past it, with plan
 * precision 1 or 2, the changes are found on the Wittrick-Williams count
 * T = s + 2 J0 (s: negative eigenvalues of K; J0: modes of the finite layers
 * with both faces clamped, counted by halving each layer's thickness), which
 * never decreases along the grid and jumps by an odd amount exactly where
 * det K changes sign: an FP32 search on T locates each rise (about log3(n_lim)
 * FP32 evaluations) and the FP64 count at V[n-1] and V[n] certifies it; where
 * the FP32 location is off, FP64 steps and the FP64 search on T take over.
 * Items whose FP64 counts fail (see masw_last_changes_linear) and plan
 * precision 0 use the FP64 scan at every grid point from one point below the
 * first change. No FP32 sign screen is used past the first change (next to a
 * pole an FP32 error can hide a root-pole pair inside one grid interval): every
 * gap between events is certified on the FP64 count. It also
 * leaves masw_dispersion's outputs of the batch updated. Runs on the batch
 * stream; synchronises it for host outputs. Device buffers of n_items x
 * max_changes are allocated on first use. MASW_EINVAL for max_changes out of
 * range. */
int masw_dispersion_changes(masw_batch* batch, int32_t max_changes, double* ct, int32_t* ct_idx,
                            int32_t* status, int32_t* delta_count, int32_t out_mem_space);

/* Items of the most recent masw_dispersion_changes call whose FP64 mode counts
 * failed (a rescaling failure, or the count not monotone at the evaluated
 * points) and that were scanned at every grid point instead; -1 when that
 * call used the plain FP64 scan (plan precision 0) or none was made.
 * Synchronises the batch stream. */
int masw_last_changes_linear(const masw_batch* batch, int32_t* n);

/* ---------------------------------------------------------------------
 * Leaky continuation. The paper builds its stiffness matrices in complex
 * arithmetic (Section 3.3) and takes the sign of their determinants
 * (Algorithm 1); masw_dispersion scans only below the half-space shear speed,
 * where K is real. This scans the whole grid.
 * --------------------------------------------------------------------- */

/* Algorithm 1 over every test velocity V[0..n_c-1] with the sign of Re det K:
 * at c >= beta_halfspace the half-space block is complex, with
 * s = i sqrt(c^2/beta^2 - 1) and r = sqrt(1 - c^2/alpha^2) or
 * i sqrt(c^2/alpha^2 - 1) in the same closed form; the finite layers stay
 * real. Taking the other root for both r and s conjugates det K, so the sign
 * of its real part does not depend on the branch. For each item: ct = V[n]
 * and ct_idx = n for the first n >= 1 whose sign differs from V[n-1]'s,
 * status MASW_FOUND; MASW_NO_ROOT (NaN, -1) when there is none on the whole
 * grid. Below beta_halfspace the sign is masw_dispersion's, so every item that
 * masw_dispersion resolves keeps its result; the others are continued in FP64
 * from the scan limit. Outputs per item in item order (host or device buffers
 * per out_mem_space, any may be NULL). Also leaves masw_dispersion's outputs
 * of the batch updated. Runs on the batch stream; synchronises it for host
 * outputs. Device buffers of n_items entries are allocated on first use
 * (MASW_ENOMEM when that fails). */
int masw_dispersion_leaky(masw_batch* batch, double* ct, int32_t* ct_idx, int32_t* status,
                          int32_t out_mem_space);

/* Items of the most recent counting-search scan (plan precision 2) that fell
 * back from the FP32 search (change above the pole-free bound, a mode below
 * V[0], or an even count jump) to the linear FP32 scan, checked like plan
 * precision 1 on the FP64 mode count; -1 for other plans. Synchronises the
 * batch stream. */
int masw_last_scan_fallback(const masw_batch* batch, int32_t* n);

/* The library's own FP64 exponential (e^x for x <= 0, a table-driven method;
 * used for e^(-k h w) in the element stiffness) and CUDA's exp at the same n
 * host points x (all <= 0, else MASW_EINVAL), into host arrays y_lib and
 * y_cuda; a diagnostic for testing its error bound. No paper counterpart.
 * Allocates and frees a device buffer of 3n doubles; synchronises
 * cuda_stream. */
int masw_exp_check(int32_t n, const double* x, double* y_lib, double* y_cuda, void* cuda_stream);

/* The library's own FP64 sine and cosine for 0 <= x < 5 pi / 4 (Cody-Waite
 * reduction by a multiple of pi/2 and Taylor series; used by the
 * clamped-layer mode count, whose arguments stay below pi) and CUDA's sincos
 * at the same n host points x (each in [0, 1.25 * 3.141592653589793], else
 * MASW_EINVAL), into host arrays s_lib, c_lib, s_cuda, c_cuda; a diagnostic
 * for testing its error. No paper counterpart. Allocates and frees a device
 * buffer of 5n doubles; synchronises cuda_stream. */
int masw_sincos_check(int32_t n, const double* x, double* s_lib, double* c_lib, double* s_cuda,
                      double* c_cuda, void* cuda_stream);

/* The element stiffness of finite layer layer[t] (0-based) of item item[t]'s
 * model at test velocity c[t] > 0, from the FP64 element and from the
 * double-float element of the counting certificate (dd_trig 0) or of the
 * leaky continuation (dd_trig 1: its trigonometric branch in double-float
 * too); a diagnostic for testing the latter's accuracy. No paper counterpart. Outputs (host arrays, 7
 * doubles per point): the common denominator and the numerators
 * (D, K11 00, K11 01, K11 11, K12 00, K12 01, K12 11) with K = numerator / D
 * in units of k (the two may scale D and the numerators by different
 * positive factors; the ratios are the element's entries). MASW_EINVAL for an
 * item or layer out of range or a non-positive c. Allocates and frees a
 * device buffer of 16 n doubles; synchronises the batch stream. */
int masw_element_check(masw_batch* batch, int32_t n, const int32_t* item, const int32_t* layer,
                       const double* c, int32_t dd_trig, double* fp64, double* df);

/* FP64 fused multiply-add throughput of this GPU in flop/s (2 per DFMA),
 * measured by a dependent-chain microbenchmark on `cuda_stream`. */
int masw_fp64_peak(void* cuda_stream, double* flops);

/* Number of streaming multiprocessors of the current device. */
int masw_sm_count(int32_t* sms);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of model evaluations. No paper counterpart
 * beyond its motivation (repeated evaluation inside an optimisation or
 * uncertainty loop, Section 1 and Section 2.1): requests, each one model
 * with its own layer count and wavelengths, arrive at any time; each
 * admitted request holds a slot with its data resident on the device. Every
 * tick uploads the requests admitted since the last one (one copy), runs the
 * counting search of plan precision 2 on their (request, wavelength) items,
 * advances every item scanning linearly (its change above the pole-free
 * bound) by at most chunks_per_tick chunks of Algorithm 1, checks in FP64
 * what these located, and compacts the rest, so requests admitted between
 * ticks overlap with those in flight. A result is identical to
 * masw_dispersion's for the same model. The host waits for a tick on an
 * event; nothing waits on the device.
 * --------------------------------------------------------------------- */
typedef struct masw_server masw_server;

typedef struct {
    int32_t max_slots;       /* requests in flight at most */
    int32_t max_layers;      /* finite layers per request (<= MASW_MAX_LAYERS) */
    int32_t max_lambda;      /* wavelengths per request */
    int64_t mem_cap_bytes;   /* admission cap on the device bytes held by requests in flight */
    int32_t chunks_per_tick; /* chunks of 64 test velocities (paired FP32 screen) an item
                                scanning linearly advances per tick */
    int32_t warps_per_block; /* 1, 2, 4 or 8 */
} masw_server_config;

typedef struct {
    int32_t in_flight;       /* slots held */
    int32_t active_items;    /* items still scanning */
    int64_t bytes_in_flight; /* bytes charged against mem_cap_bytes */
    int64_t ticks;
    int64_t completed;
} masw_server_stats;

/* Allocate the slot table (device), its packed upload buffer (pinned host and
 * device, one slot block per slot) and the mapped result buffers for the
 * given grid; all later work runs on cuda_stream. MASW_EINVAL on a bad config
 * (including an upload buffer above 2^31 bytes), MASW_ENOMEM when the
 * buffers do not fit. */
int masw_server_create(const masw_grid* grid, const masw_server_config* cfg, void* cuda_stream,
                       masw_server** out);
int masw_server_destroy(masw_server* server);

/* Admit one request (host arrays as in masw_models_desc for one model).
 * MASW_EADMIT when no slot is free or its bytes would exceed the cap (the
 * server is unchanged; retry after a tick); MASW_EINVAL on invalid values.
 * The request joins the next tick. */
int masw_server_submit(masw_server* server, int32_t n_layers, const double* h,
                       const double* alpha, const double* beta, const double* rho,
                       int32_t n_lambda, const double* lambda, int64_t* request_id);

/* Run one tick and wait for it; *n_completed = requests that finished. */
int masw_server_tick(masw_server* server, int32_t* n_completed);

/* Copy a finished request's results (host arrays of its n_lambda entries,
 * any may be NULL) and free its slot; MASW_EAGAIN if not finished yet. */
int masw_server_poll(masw_server* server, int64_t request_id, double* ct, int32_t* ct_idx,
                     int32_t* status);

int masw_server_get_stats(const masw_server* server, masw_server_stats* stats);

/* Test routing of the server's scan, as masw_set_route: 1 every new item
 * takes the linear FP32 screen from V[0]; 2 also fails every three-point FP64
 * check (mode-count search); 3 also sends every searched item to the FP64
 * scan from V[0], one chunk per tick. Applies from the next tick; results must
 * not change. MASW_EINVAL outside 0..3. */
int masw_server_set_route(masw_server* server, int32_t route);

/* Opt-in profile of the server's ticks, for measurement: enable = 1 starts
 * it (zeroing the totals; it waits for the server's stream once), 0 stops
 * it; out (may be NULL) receives MASW_SERVER_PROFILE_VALUES totals:
 *   [0] ticks profiled;
 *   device milliseconds (CUDA events between the parts of each tick):
 *   [1] upload and scatter of the newly admitted requests, [2] count kernel
 *   (counting search + certificate of the new items), [3] tick kernel (linear
 *   FP32 chunks), [4] check kernel, [5] read-back of counters and done list;
 *   host milliseconds: [6] launching ticks (staging included), [7] finishing
 *   ticks (the wait for the tick's event included), [8] admitting requests
 *   (masw_server_submit). While on, every tick records six more events. */
#define MASW_SERVER_PROFILE_VALUES 9
int masw_server_profile(masw_server* server, int32_t enable, double* out);

/* Replay a request trace natively: request i (concatenated host arrays as in
 * masw_models_desc) arrives arrival_s[i] seconds (non-decreasing) after the
 * call starts; the loop admits arrived requests while slots and bytes allow,
 * ticks, and retires finished ones. latency_s[i] = completion - arrival.
 * ct, ct_idx, status (sum of n_lambda, may be NULL) receive the results;
 * stats (3 values, may be NULL): ticks, refused admissions, max in flight.
 * The server must be idle. MASW_ETIMEOUT after timeout_s seconds. */
int masw_server_run_trace(masw_server* server, int32_t n_requests, const int32_t* n_layers,
                          const double* h, const double* alpha, const double* beta,
                          const double* rho, const int32_t* n_lambda, const double* lambda,
                          const double* arrival_s, double timeout_s, double* latency_s,
                          double* ct, int32_t* ct_idx, int32_t* status, int64_t* stats);

/* Algorithm 1 for callers that cannot allocate memory. The paper has no
 * counterpart: this exists for embedders whose GPU memory is handed out by
 * someone else (a framework allocator, a fixed budget, a service that forbids
 * allocation after start-up), so masw_model_batch_create, which allocates a
 * device copy of the batch, is not open to them. This call allocates nothing,
 * neither on the device nor on the host: everything derived from the inputs
 * (layer records in FP64, FP32 and double-float, offsets, scan limits,
 * wavenumbers, item order, the counting search's per-item lists and
 * counters) goes to one fixed array of MASW_NOALLOC_SCRATCH_BYTES (5.3 MiB)
 * in device memory that every GPU loading the library holds until exit.
 *  - models: like masw_model_batch_create (host or device arrays, mem_space);
 *    grid as there. Every input array must lie in the space mem_space
 *    declares (device or managed memory for MASW_DEVICE, host memory for
 *    MASW_HOST); a mixed call returns MASW_EINVAL before any copy or launch.
 *    ct, ct_idx, status: DEVICE buffers of sum(n_lambda) entries, same
 *    meaning as masw_dispersion; results equal its results.
 *  - It runs masw_dispersion's default counting plan in the form that plan
 *    takes for batches of this size (the fused search and certificate, then
 *    the fallback chain), with the same indices.
 *  - Limits: n_models <= MASW_NOALLOC_MAX_MODELS, sum(N_m + 1) <=
 *    MASW_NOALLOC_MAX_RECORDS, sum(n_lambda) <= MASW_NOALLOC_MAX_ITEMS;
 *    beyond them the call returns MASW_ETOOBIG and touches nothing.
 *  - The first call on a device looks up the array's device address (once,
 *    with that device current).
 *  - Every call validates on the GPU and waits for that check: it copies an
 *    error word to the host and synchronises cuda_stream before it launches
 *    the scan, then enqueues the scan and returns; the outputs are complete
 *    when cuda_stream reaches that point. Because of that synchronisation no
 *    call may be made while a stream capture is under way.
 *  - All calls share the one array and every call overwrites it: calls that
 *    may run at the same time on the GPU (other streams, other threads) race
 *    and give wrong results. Calls on one stream are ordered and safe. */
#define MASW_NOALLOC_MAX_MODELS 1024
#define MASW_NOALLOC_MAX_RECORDS 16384
#define MASW_NOALLOC_MAX_ITEMS 65536
#define MASW_NOALLOC_SCRATCH_BYTES 5518592
int masw_dispersion_noalloc(const masw_models_desc* models, const masw_grid* grid,
                            void* cuda_stream, double* ct, int32_t* ct_idx, int32_t* status);

const char* masw_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MASW_H */
