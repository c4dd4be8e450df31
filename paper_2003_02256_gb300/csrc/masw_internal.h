// masw_internal.h -- device-side data layout and kernel launchers shared by
// the C-ABI layer (masw_api.cu) and the kernels (masw_kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace masw {

// Device view of a ragged model batch.
struct DevBatch {
    const double* layers;      // [n_records][LAYER_STRIDE] records, per model N finite + 1 half-space
    const float* layers_df;    // [n_records][LAYER_STRIDE_DF] double-float records of the same
                               // layers (counting certificate), or nullptr: split on the fly
    const int32_t* model_loff; // [n_models + 1] record offsets
    const int32_t* model_nlim; // [n_models] number of grid points below beta_halfspace
    const int32_t* model_woff; // [n_models + 1] item offsets (items of model m are contiguous)
    const double* k;           // [n_items] wavenumber 2*pi/lambda
    const int32_t* item_model; // [n_items]
    const int32_t* order;      // [n_items] item ids in processing order
    const int64_t* grad_off;   // [n_items + 1] offsets of per-item gradient rows (2N+1 each)
    int32_t n_models;
    int32_t n_items;
    double c0, dc;
    int32_t n_c;
    int32_t route;  // test routing (masw_set_route): 0 normal, 1..3 force the slower paths,
                    // 4 displaces the FP32-located higher-mode events
    // the split counting search's two passes (or nullptr: one pass): item ids,
    // model by model from the most layers down, first the n_anchor items
    // searched in full (every SEARCH_STRIDE-th item of a model and its last),
    // then the others, bracketed by those neighbours
    const int32_t* search_order = nullptr;
    int32_t n_anchor = 0;
    // all items, model by model from the fewest layers up (the split
    // certificate's order over a whole batch), or nullptr
    const int32_t* layer_order = nullptr;
};

// Items of a model between two fully searched ones in the split search.
constexpr int SEARCH_STRIDE = 6;

// The cumulative level 0..3 of a test routing value (route 4 has none).
__host__ __device__ inline int route_level(int route) { return route <= 3 ? route : 0; }

// Test routing 4: grid points by which the higher-mode search displaces an
// item's FP32-located events before their FP64 certificate (by item % 5), so
// that every recovery branch runs.
__host__ __device__ inline int route_displacement(int route, int item) {
    if (route != 4) return 0;
    const int d[5] = {0, -1, 1, 3, -7};
    return d[item % 5];
}

struct ScanOut {
    double* ct;
    int32_t* idx;
    int32_t* status;
    // counting kernel (or nullptr): per item PairCount::counts, the FP64
    // counts of the certificate, -1 when the item was not certified in the
    // pole-free range
    int32_t* cert_counts = nullptr;
};

// Launch configuration of the scan (the batch plan).
struct ScanPlan {
    int warps_per_block;  // 1..32
    int cpl;              // test velocities per lane per chunk: 1, 2 or 4
    int blocks;           // grid size (persistent: multiple of the SM count)
    int persistent;       // 1: warps pop items from a queue; 0: one item per warp
    int stage_layers;     // layer records staged in shared memory per warp (0 = read global)
    int count_block = 128;  // threads per block of the counting kernel: 64, 128 or 256
    int count_split = 0;    // 1: the counting search in a kernel of its own; 2: as 1, and
                            // the search's fallback items on a second stream (ScanSide)
    int sms = 0;            // SM count (0: unknown)
};

// FP32 screen + FP64 decision (masw_screen.cuh, masw_kernels.cu). counting
// 0: linear FP32 screen; 1: counting search with the linear screen as
// fallback. Both check on the FP64 mode count and search it for the items
// that fail. n32, search, unresolved, fallback: n_items each; counters:
// SCAN_COUNTERS per list set ([3]: fallback items, [5]: items that failed
// their FP64 check).
constexpr int SCAN_COUNTERS = 7;
// n32 flag of an index located by the counting search (MASW_SCREEN_COUNTED)
constexpr int32_t SCREEN_COUNTED = 1 << 30;
// Plan count_split 2: a second stream for the items the counting search
// passes straight to the linear FP32 scan. After the search kernel, `fork` on
// the scan stream releases that stream; its fallback scan, check, mode-count
// search and re-scan run (at priority `prio`, the stream's) beside the
// certificate over lists of their own, and the scan stream waits for `join`
// at the end. nsearch, search, unresolved, fallback: n_items each.
struct ScanSide {
    cudaStream_t s;
    int prio;
    cudaEvent_t fork, join;
    int32_t* nsearch;  // the search kernel's index per item (0: passed on)
    int32_t* search;
    int32_t* unresolved;
    int32_t* fallback;
};
// counters: 2 x SCAN_COUNTERS (the second set for the side stream's lists).
cudaError_t launch_screen_scan(const DevBatch& b, const ScanOut& o, const ScanPlan& p,
                               const float* layers32, int32_t* n32, int32_t* search,
                               int32_t* unresolved, int32_t* fallback, int32_t* counters,
                               int counting, int item_begin, int item_end, cudaStream_t s,
                               cudaEvent_t* phase_ev,  // nullptr or 3 events
                               const ScanSide* side);  // nullptr: one stream

// Algorithm 1 continued: the first M sign changes per item with their
// negative-eigenvalue count changes, from the first change `first` (the batch
// scan's index, -1: none); outputs [n_items][M]. counting 0: FP64 linear scan
// from one point below it; 1: FP64 search on the monotone mode count
// s + 2 J0, items whose counts fail going to the linear scan (linear:
// n_items entries). counters: CHANGES_COUNTERS, [1] = linear-scan items
// (masw_kernels.cu).
constexpr int CHANGES_COUNTERS = 2;
cudaError_t launch_changes(const DevBatch& b, const ScanPlan& p, int M, const int32_t* first,
                           const int32_t* cert_counts, const float* layers32, double* ct, int32_t* idx, int32_t* status,
                           int32_t* delta, int32_t* counters, int32_t* linear, int counting,
                           cudaStream_t s);

// Leaky continuation: Algorithm 1 over the whole grid with the sign of Re det K
// (complex half-space block at c >= beta_hs); items the batch scan resolved
// (status_in 0) keep idx_in; outputs o; work: 2 n_items + 4; dd: the scan in
// double-float (det_sign_leaky_df), each change confirmed with the FP64 step
// and the unconfirmed items scanned again in FP64; else the FP64 scan
// (masw_kernels.cu).
cudaError_t launch_leaky(const DevBatch& b, const ScanPlan& p, const int32_t* idx_in,
                         const int32_t* status_in, const ScanOut& o, int32_t* work, int dd,
                         cudaStream_t s);

cudaError_t launch_scan(const DevBatch& b, const ScanOut& o, const ScanPlan& p, int32_t* counter,
                        int item_begin, int item_end, cudaStream_t s);
cudaError_t launch_det_eval(const DevBatch& b, int n, const int32_t* item, const double* c,
                            int32_t* sign, double* log_abs, cudaStream_t s);
cudaError_t launch_mode_count(const DevBatch& b, int n, const int32_t* item, const double* c,
                              int32_t* s, int32_t* j0, cudaStream_t st);
cudaError_t launch_refine(const DevBatch& b, const int32_t* idx, double rel_tol, double* croot,
                          cudaStream_t s);
cudaError_t launch_root_grad(const DevBatch& b, const double* croot, double* rows, double* bs,
                             cudaStream_t s);
cudaError_t launch_misfit(const DevBatch& b, const double* ct, const double* ce, int kind,
                          double sigma, double* misfit, double* dphi_dc, cudaStream_t s);
cudaError_t launch_grad_reduce(const DevBatch& b, const double* rows, const double* dphi_dc,
                               double* grad_beta, double* grad_h, cudaStream_t s);
// Model update on the device: validation flag in err (which must start at 0),
// then records and scan limits unless it was set (masw_kernels.cu).
cudaError_t launch_model_update(const DevBatch& b, const double* h, const double* alpha,
                                const double* beta, const double* rho, double* layers,
                                float* layers32, float* layers_df, int32_t* nlim, int32_t* err,
                                cudaStream_t s);
cudaError_t launch_update_beta_h(const DevBatch& b, const double* h, const double* beta,
                                 double* layers, float* layers32, float* layers_df, int32_t* nlim,
                                 int32_t* err, cudaStream_t s);
cudaError_t launch_element_check(const DevBatch& b, int n, const int32_t* item, const int32_t* layer,
                                 const double* c, int dd_trig, double* fp64, double* df,
                                 cudaStream_t s);
cudaError_t launch_exp_check(int n, const double* x, double* y_lib, double* y_cuda,
                             cudaStream_t s);
cudaError_t launch_sincos_check(int n, const double* x, double* s_lib, double* c_lib,
                                double* s_cuda, double* c_cuda, cudaStream_t s);
cudaError_t launch_fp64_peak(int blocks, int threads, int iters, double* sink, cudaStream_t s);

}  // namespace masw
