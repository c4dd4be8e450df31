// masw_api.cu -- the C ABI of libmasw (include/masw.h): batch state, input
// validation, device layout, launch plans, CUDA-graph replay and autotuning.
//
// Device layout of a batch (all batch-owned, allocated once at create):
//   layers      [records][8] f64: h, mu = rho beta^2, rho, 1/alpha^2,
//               1/beta^2, beta, alpha/beta, 0 (one 64-byte line per layer;
//               each model has N finite records then its half-space)
//   model_loff  [M+1] i32 record offsets;  model_woff [M+1] i32 item offsets
//   model_nlim  [M] i32 grid points below the half-space shear speed
//   k           [items] f64 2 pi / lambda;  item_model [items] i32
//   order       [items] i32 processing order (longest predicted scan first)
//   ct, idx, status [items] results of the last scan
//   FP32 records, screen indices, the search / re-scan / fallback lists and
//   their counters (two-precision plans)
// plus lazily allocated buffers for roots, gradient rows and misfits, model
// updates, the higher modes and the leaky continuation.
#include <algorithm>
#include <functional>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/masw.h"
#include "masw_device.cuh"
#include "masw_df.cuh"
#include "masw_internal.h"
#include "masw_screen.cuh"

using namespace masw;

struct masw_batch {
    int32_t n_models = 0;
    int64_t n_items = 0;
    int64_t n_records = 0;
    int32_t max_layers = 0;
    int64_t grad_len = 0;
    masw_grid grid{};
    cudaStream_t stream = nullptr;
    int sm_count = 0;

    // nlim: scan limits at creation, for the processing order only (updates
    // rebuild the device copy, d_nlim)
    std::vector<int32_t> n_layers, n_lambda, loff, woff, nlim, item_model;
    std::vector<double> lambda, kvec;
    std::vector<int32_t> order_sorted, order_natural;
    std::vector<int32_t> search_order;  // anchors of the split search, then the others
    std::vector<int32_t> layer_order;   // items by model, models ordered by layer count
    int32_t n_anchor = 0;
    std::vector<int64_t> grad_off;

    double* d_layers = nullptr;
    int32_t* d_loff = nullptr;
    int32_t* d_woff = nullptr;
    int32_t* d_nlim = nullptr;
    double* d_k = nullptr;
    int32_t* d_item_model = nullptr;
    int32_t* d_order_sorted = nullptr;
    int32_t* d_order_natural = nullptr;
    int32_t* d_search_order = nullptr;
    int32_t* d_layer_order = nullptr;
    int64_t* d_grad_off = nullptr;
    int32_t* d_counter = nullptr;
    double* d_ct = nullptr;
    int32_t* d_idx = nullptr;
    int32_t* d_status = nullptr;
    // lazily allocated
    double* d_croot = nullptr;
    double* d_rows = nullptr;
    double* d_bs = nullptr;
    double* d_dphi = nullptr;
    double* d_ce = nullptr;
    double* d_misfit = nullptr;
    double* d_gb = nullptr;
    double* d_gh = nullptr;
    // two-precision scan
    float* d_layers32 = nullptr;
    float* d_layers_df = nullptr;  // double-float records of the counting certificate
    int32_t* d_n32 = nullptr;
    int32_t* d_cert = nullptr;  // per item: the counting certificate's FP64 counts (ScanOut)
    int32_t* d_search = nullptr;
    int32_t* d_unres = nullptr;
    int32_t* d_fallback = nullptr;
    int32_t* d_counters = nullptr;  // 2 x SCAN_COUNTERS (scan stream's lists, side stream's)
    // plan count_split 2: the search's fallback items on a second stream
    cudaStream_t side = nullptr;
    int side_prio = 0;
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    int32_t* d_nsearch = nullptr;
    int32_t* d_search2 = nullptr;
    int32_t* d_unres2 = nullptr;
    int32_t* d_fallback2 = nullptr;
    // model updates (allocated on first use): staged host arrays, error flag
    double* d_upd = nullptr;
    int32_t* d_upd_err = nullptr;
    // higher modes (allocated on first use, for chg_cap changes per item)
    int chg_cap = 0;
    double* d_chg_ct = nullptr;
    int32_t* d_chg_idx = nullptr;
    int32_t* d_chg_status = nullptr;
    int32_t* d_chg_delta = nullptr;
    int32_t* d_chg_counters = nullptr;  // CHANGES_COUNTERS, then an n_items list
    bool changes_counted = false;
    // leaky continuation (allocated on first use): per-item outputs, counter
    double* d_lk_ct = nullptr;
    int32_t* d_lk_idx = nullptr;  // [n_items] idx, [n_items] status, then 2 n_items + 4 of work
    masw_plan plan{};
    int32_t route = 0;  // masw_set_route
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t phase_ev[3] = {nullptr, nullptr, nullptr};  // after: counting, search, (split) FP32 search
    bool phases_valid = false;
    bool count_phases_valid = false;  // phase_ev[2] recorded (split counting kernels)
    bool side_phase_valid = false;    // side_fork / side_join recorded (count_split 2)
    float last_ms = 0.f;

    DevBatch dev(bool ordered) const {
        DevBatch b;
        b.layers = d_layers;
        b.layers_df = d_layers_df;
        b.model_loff = d_loff;
        b.model_nlim = d_nlim;
        b.model_woff = d_woff;
        b.k = d_k;
        b.item_model = d_item_model;
        b.order = ordered ? d_order_sorted : d_order_natural;
        b.search_order = d_search_order;
        b.layer_order = d_layer_order;
        b.n_anchor = n_anchor;
        b.grad_off = d_grad_off;
        b.n_models = n_models;
        b.n_items = (int32_t)n_items;
        b.c0 = grid.c0;
        b.dc = grid.dc;
        b.n_c = grid.n_c;
        b.route = route;
        return b;
    }
};

// ------------------------------------------------------------- helpers

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) {                \
            record_cuda_error(e_, #x, __LINE__); \
            return MASW_ECUDA;                  \
        }                                       \
    } while (0)

static thread_local char g_last_cuda[256] = "";

static void record_cuda_error(cudaError_t e, const char* what, int line) {
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s (%s) at masw_api.cu:%d", cudaGetErrorString(e),
             what, line);
}

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// masw_test_fail_alloc: ordinal of the next device allocation to fail (-1: none)
static std::atomic<int> g_alloc_fail_at{-1};

template <typename T>
static int dev_alloc(T** p, size_t n) {
    // test hook (masw_test_fail_alloc): the allocation with this ordinal fails
    const int at = g_alloc_fail_at.load();
    if (at >= 0) {
        g_alloc_fail_at.store(at - 1);
        if (at == 0) {
            *p = nullptr;
            return MASW_ENOMEM;
        }
    }
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return MASW_ENOMEM;
    }
    return MASW_OK;
}

template <typename T>
static int fetch(std::vector<T>& dst, const T* src, size_t n, bool device) {
    dst.resize(n);
    if (n == 0) return MASW_OK;
    if (!src) return MASW_EINVAL;
    if (device) {
        CK(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(dst.data(), src, n * sizeof(T));
    }
    return MASW_OK;
}

// Copy n elements from a batch buffer to a caller buffer (host or device).
template <typename T>
static int copy_out(T* dst, const T* src, size_t n, cudaStream_t s, bool* need_sync) {
    if (!dst || n == 0) return MASW_OK;
    if (is_device_ptr(dst)) {
        CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyDeviceToHost, s));
        *need_sync = true;
    }
    return MASW_OK;
}

template <typename T>
static int copy_in(T* dst, const T* src, size_t n, cudaStream_t s) {
    if (n == 0) return MASW_OK;
    if (!src) return MASW_EINVAL;
    cudaMemcpyKind kind = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(dst, src, n * sizeof(T), kind, s));
    if (kind == cudaMemcpyHostToDevice) CK(cudaStreamSynchronize(s));  // caller may reuse src
    return MASW_OK;
}

static double grid_v(const masw_grid& g, int n) { return std::fma((double)n, g.dc, g.c0); }

// Number of grid points with V[n] < beta_hs (same rounding as the device).
static int32_t scan_limit(const masw_grid& g, double beta_hs) {
    double est = std::floor((beta_hs - g.c0) / g.dc);
    int64_t n = (int64_t)std::max(0.0, std::min(est, (double)g.n_c));
    while (n > 0 && !(grid_v(g, (int)(n - 1)) < beta_hs)) --n;
    while (n < g.n_c && grid_v(g, (int)n) < beta_hs) ++n;
    return (int32_t)n;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

static int validate_layers(const int32_t* nl, size_t n_models, const double* h, const double* a,
                           const double* b, const double* r) {
    size_t ih = 0, il = 0;
    for (size_t m = 0; m < n_models; ++m) {
        for (int i = 0; i < nl[m]; ++i)
            if (!finite_pos(h[ih++])) return MASW_EINVAL;
        for (int i = 0; i <= nl[m]; ++i, ++il) {
            if (!finite_pos(a[il]) || !finite_pos(b[il]) || !finite_pos(r[il])) return MASW_EINVAL;
            // positive bulk modulus: alpha^2 > 4/3 beta^2 (also keeps r != s)
            if (!(3.0 * a[il] * a[il] > 4.0 * b[il] * b[il])) return MASW_EINVAL;
        }
    }
    return MASW_OK;
}

static int validate_layers(const std::vector<int32_t>& nl, const std::vector<double>& h,
                           const std::vector<double>& a, const std::vector<double>& b,
                           const std::vector<double>& r) {
    return validate_layers(nl.data(), nl.size(), h.data(), a.data(), b.data(), r.data());
}

static void build_records(masw_batch* B, const std::vector<double>& h, const std::vector<double>& a,
                          const std::vector<double>& b, const std::vector<double>& r,
                          std::vector<double>& rec) {
    rec.assign((size_t)B->n_records * LAYER_STRIDE, 0.0);
    size_t ih = 0, il = 0;
    for (int32_t m = 0; m < B->n_models; ++m) {
        int N = B->n_layers[m];
        for (int i = 0; i <= N; ++i, ++il) {
            double* L = &rec[il * LAYER_STRIDE];
            L[L_H] = (i < N) ? h[ih++] : 0.0;
            L[L_MU] = r[il] * b[il] * b[il];
            L[L_RHO] = r[il];
            L[L_IA2] = 1.0 / (a[il] * a[il]);
            L[L_IB2] = 1.0 / (b[il] * b[il]);
            L[L_BETA] = b[il];
            L[L_RATIO] = a[il] / b[il];
            L[L_IRHO] = 1.0 / r[il];
        }
    }
}

// FP32 records of the screen: stiffnesses divided by the half-space shear
// modulus of the model (a positive common factor).
static void build_records32(const masw_batch* B, const std::vector<double>& rec,
                            std::vector<float>& rec32) {
    rec32.assign((size_t)B->n_records * LAYER_STRIDE32, 0.0f);
    for (int32_t m = 0; m < B->n_models; ++m) {
        int lo = B->loff[m], N = B->n_layers[m];
        double mref = rec[(size_t)(lo + N) * LAYER_STRIDE + L_MU];
        for (int i = 0; i <= N; ++i) {
            const double* L = &rec[(size_t)(lo + i) * LAYER_STRIDE];
            float* F = &rec32[(size_t)(lo + i) * LAYER_STRIDE32];
            F[F_H] = (float)L[L_H];
            F[F_MU] = (float)(L[L_MU] / mref);
            F[F_RHO] = (float)(L[L_RHO] / mref);
            F[F_IA2] = (float)L[L_IA2];
            F[F_IB2] = (float)L[L_IB2];
            F[F_DIB] = (float)(L[L_IB2] - L[L_IA2]);
        }
    }
}

// Predicted scan length of an item (speed only): the first root sits near
// 0.93 x the shear speed at depth ~ lambda/2.
static double predicted_cost(const masw_batch* B, int32_t m, double lam,
                             const std::vector<double>& h, const std::vector<double>& b,
                             size_t h0, size_t l0) {
    int N = B->n_layers[m];
    double depth = 0.5 * lam, z = 0.0, be = b[l0 + N];
    for (int i = 0; i < N; ++i) {
        z += h[h0 + i];
        if (z >= depth) { be = b[l0 + i]; break; }
    }
    double n = (0.93 * be - B->grid.c0) / B->grid.dc;
    n = std::max(1.0, std::min(n, (double)B->nlim[m]));
    return (n + 32.0) * (N + 1);
}

static void free_batch(masw_batch* B) {
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->ev0) cudaEventDestroy(B->ev0);
    if (B->ev1) cudaEventDestroy(B->ev1);
    for (cudaEvent_t e : B->phase_ev)
        if (e) cudaEventDestroy(e);
    if (B->side_fork) cudaEventDestroy(B->side_fork);
    if (B->side_join) cudaEventDestroy(B->side_join);
    if (B->side) cudaStreamDestroy(B->side);
    void* ptrs[] = {B->d_layers, B->d_loff,  B->d_woff,  B->d_nlim,   B->d_k,
                    B->d_item_model, B->d_order_sorted, B->d_order_natural, B->d_search_order,
                    B->d_layer_order,
                    B->d_grad_off,
                    B->d_counter, B->d_ct, B->d_idx, B->d_status, B->d_croot, B->d_rows, B->d_bs,
                    B->d_dphi, B->d_ce, B->d_misfit, B->d_gb, B->d_gh, B->d_layers32, B->d_layers_df,
                    B->d_n32, B->d_cert, B->d_search, B->d_unres, B->d_fallback, B->d_counters,
                    B->d_nsearch, B->d_search2, B->d_unres2, B->d_fallback2, B->d_upd, B->d_upd_err,
                    B->d_chg_ct, B->d_chg_idx, B->d_chg_status, B->d_chg_delta,
                    B->d_chg_counters, B->d_lk_ct, B->d_lk_idx};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete B;
}

static_assert(MASW_SCREEN_COUNTED == SCREEN_COUNTED, "n32 flag of the counting search");

static masw_plan default_plan(const masw_batch* B) {
    masw_plan p;
    p.warps_per_block = 8;
    p.cpl = 2;
    p.blocks_per_sm = 4;
    p.persistent = 1;
    p.ordered = 1;
    p.stage_layers = std::min(B->max_layers + 1, 32);
    p.use_graph = 1;
    p.precision = 2;
    // the fused kernel's lane pairs give small batches the shortest chain;
    // large ones take the split kernels, and from a quarter million items
    // the search's fallback items on the second stream
    p.count_split = B->n_items < (1 << 17) ? 0 : B->n_items < (1 << 18) ? 1 : 2;
    // beside the second stream's chain the certificate runs in blocks of 256
    // (512 resident threads per SM, against 896 in blocks of 128: measured
    // faster there, the chain ending sooner), else of 128
    p.count_block = p.count_split == 2 ? 256 : 128;
    return p;
}

static bool plan_ok(const masw_plan& p) {
    bool wpb = p.warps_per_block == 1 || p.warps_per_block == 2 || p.warps_per_block == 4 ||
               p.warps_per_block == 8;
    bool cpl = p.cpl == 1 || p.cpl == 2 || p.cpl == 4;
    bool cb = p.count_block == 64 || p.count_block == 128 || p.count_block == 256;
    bool cs = p.count_split >= 0 && p.count_split <= 2;
    return wpb && cpl && cb && cs && p.precision >= 0 && p.precision <= 2 && p.blocks_per_sm >= 1 &&
           p.blocks_per_sm <= 32 && p.stage_layers >= 0 &&
           p.stage_layers <= MASW_MAX_LAYERS + 1 &&
           (size_t)p.warps_per_block * p.stage_layers * LAYER_STRIDE * sizeof(double) <= 48 * 1024;
}

static ScanPlan to_scan_plan(const masw_batch* B, const masw_plan& p) {
    ScanPlan s;
    s.warps_per_block = p.warps_per_block;
    s.cpl = p.cpl;
    s.blocks = p.blocks_per_sm * B->sm_count;
    s.persistent = p.persistent;
    s.stage_layers = p.stage_layers;
    s.count_block = p.count_block;
    s.count_split = p.count_split;
    s.sms = B->sm_count;
    return s;
}

// Enqueue one full scan (all items) with the given plan on stream s.
static cudaError_t enqueue_scan(masw_batch* B, const masw_plan& p, cudaStream_t s,
                                bool phase_events = false) {
    if (p.precision >= 1) {
        ScanOut o{B->d_ct, B->d_idx, B->d_status, B->d_cert};
        ScanSide side{B->side, B->side_prio, B->side_fork, B->side_join,
                      B->d_nsearch, B->d_search2, B->d_unres2, B->d_fallback2};
        return launch_screen_scan(B->dev(p.ordered != 0), o, to_scan_plan(B, p), B->d_layers32,
                                  B->d_n32, B->d_search, B->d_unres, B->d_fallback, B->d_counters,
                                  p.precision == 2, 0, (int)B->n_items, s,
                                  phase_events ? B->phase_ev : nullptr,
                                  p.precision == 2 && p.count_split == 2 ? &side : nullptr);
    }
    if (p.persistent) {
        cudaError_t e = cudaMemsetAsync(B->d_counter, 0, sizeof(int32_t), s);
        if (e != cudaSuccess) return e;
    }
    ScanOut o{B->d_ct, B->d_idx, B->d_status};
    return launch_scan(B->dev(p.ordered != 0), o, to_scan_plan(B, p), B->d_counter, 0,
                       (int)B->n_items, s);
}

static int rebuild_graph(masw_batch* B) {
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    if (!B->plan.use_graph) return MASW_OK;
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = enqueue_scan(B, B->plan, cap);
        e = cudaStreamEndCapture(cap, &g);
        if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) {
        // the side stream's kernels keep their launch priority in the graph
        e = cudaGraphInstantiateWithFlags(&B->graph, g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cap);
    CK(e);
    return MASW_OK;
}

// Run Algorithm 1 over the whole batch into the batch-owned outputs.
static int run_scan(masw_batch* B) {
    CK(cudaEventRecord(B->ev0, B->stream));
    if (B->plan.use_graph && B->graph) {
        CK(cudaGraphLaunch(B->graph, B->stream));
        B->phases_valid = false;
        B->count_phases_valid = false;
        B->side_phase_valid = false;
    } else {
        bool ph = B->plan.precision >= 1;
        CK(enqueue_scan(B, B->plan, B->stream, ph));
        B->phases_valid = ph;
        B->count_phases_valid = ph && B->plan.precision == 2 && B->plan.count_split >= 1;
        B->side_phase_valid = B->count_phases_valid && B->plan.count_split == 2;
    }
    CK(cudaEventRecord(B->ev1, B->stream));
    return MASW_OK;
}

static int ensure(double** p, size_t n) { return *p ? MASW_OK : dev_alloc(p, n); }

// ------------------------------------------------------------- the ABI

extern "C" {

const char* masw_strerror(int code) {
    switch (code) {
        case MASW_OK: return "ok";
        case MASW_EINVAL: return "invalid argument or model";
        case MASW_ENOMEM: return "out of memory";
        case MASW_EADMIT: return "request refused by the admission cap";
        case MASW_ECUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA runtime error";
        case MASW_ETIMEOUT: return "bounded wait timed out";
        case MASW_EAGAIN: return "result not ready";
        case MASW_ETOOBIG:
            return "batch exceeds the fixed scratch of masw_dispersion_noalloc (see MASW_NOALLOC_MAX_*)";
        default: return "unknown error code";
    }
}

int masw_sm_count(int32_t* sms) {
    if (!sms) return MASW_EINVAL;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int n = 0;
    CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    *sms = n;
    return MASW_OK;
}

int masw_model_batch_create(const masw_models_desc* md, const masw_grid* grid, void* cuda_stream,
                            masw_batch** out) {
    if (!md || !grid || !out) return MASW_EINVAL;
    if (md->n_models < 1 || (md->mem_space != MASW_HOST && md->mem_space != MASW_DEVICE))
        return MASW_EINVAL;
    if (!(std::isfinite(grid->c0) && grid->c0 > 0.0 && std::isfinite(grid->dc) && grid->dc > 0.0 &&
          grid->n_c >= 2))
        return MASW_EINVAL;
    bool dev = md->mem_space == MASW_DEVICE;
    masw_batch* B = new (std::nothrow) masw_batch();
    if (!B) return MASW_ENOMEM;
    B->grid = *grid;
    B->stream = (cudaStream_t)cuda_stream;
    B->n_models = md->n_models;
    int rc;
    if ((rc = fetch(B->n_layers, md->n_layers, md->n_models, dev)) ||
        (rc = fetch(B->n_lambda, md->n_lambda, md->n_models, dev))) {
        free_batch(B);
        return rc;
    }
    int64_t nh = 0, nl = 0, nw = 0;
    for (int32_t m = 0; m < B->n_models; ++m) {
        if (B->n_layers[m] < 0 || B->n_layers[m] > MASW_MAX_LAYERS || B->n_lambda[m] < 0) {
            free_batch(B);
            return MASW_EINVAL;
        }
        nh += B->n_layers[m];
        nl += B->n_layers[m] + 1;
        nw += B->n_lambda[m];
        B->max_layers = std::max(B->max_layers, B->n_layers[m]);
    }
    if (nw > INT32_MAX / 2 || nl > INT32_MAX / 2) {
        free_batch(B);
        return MASW_EINVAL;
    }
    B->n_records = nl;
    B->n_items = nw;
    std::vector<double> h, a, b, r;
    if ((rc = fetch(h, md->h, nh, dev)) || (rc = fetch(a, md->alpha, nl, dev)) ||
        (rc = fetch(b, md->beta, nl, dev)) || (rc = fetch(r, md->rho, nl, dev)) ||
        (rc = fetch(B->lambda, md->lambda, nw, dev))) {
        free_batch(B);
        return rc;
    }
    if ((rc = validate_layers(B->n_layers, h, a, b, r))) {
        free_batch(B);
        return rc;
    }
    for (double lam : B->lambda)
        if (!finite_pos(lam)) {
            free_batch(B);
            return MASW_EINVAL;
        }
    // offsets, limits, items
    B->loff.assign(B->n_models + 1, 0);
    B->woff.assign(B->n_models + 1, 0);
    B->nlim.assign(B->n_models, 0);
    std::vector<size_t> hoff(B->n_models + 1, 0);
    for (int32_t m = 0; m < B->n_models; ++m) {
        B->loff[m + 1] = B->loff[m] + B->n_layers[m] + 1;
        B->woff[m + 1] = B->woff[m] + B->n_lambda[m];
        hoff[m + 1] = hoff[m] + B->n_layers[m];
        B->nlim[m] = scan_limit(B->grid, b[B->loff[m + 1] - 1]);
    }
    B->item_model.resize(nw);
    B->kvec.resize(nw);
    B->grad_off.assign(nw + 1, 0);
    std::vector<double> cost(nw);
    for (int32_t m = 0; m < B->n_models; ++m)
        for (int32_t j = B->woff[m]; j < B->woff[m + 1]; ++j) {
            B->item_model[j] = m;
            B->kvec[j] = 2.0 * M_PI / B->lambda[j];
            B->grad_off[j + 1] = B->grad_off[j] + 2 * B->n_layers[m] + 1;
            cost[j] = predicted_cost(B, m, B->lambda[j], h, b, hoff[m], B->loff[m]);
        }
    B->grad_len = B->grad_off[nw];
    B->order_natural.resize(nw);
    std::iota(B->order_natural.begin(), B->order_natural.end(), 0);
    // the split search: every SEARCH_STRIDE-th wavelength of a model and its
    // last are searched in full first, the items between them after. Both
    // lists run model by model, so that a warp's items (consecutive
    // wavelengths of one model, or of models with as many layers) take the
    // same number of layer steps, the models with the most layers first: the
    // longest threads start in the first wave, and the last waves, with the
    // shortest, end closer together.
    std::vector<int32_t> by_layers(B->n_models);
    std::iota(by_layers.begin(), by_layers.end(), 0);
    std::stable_sort(by_layers.begin(), by_layers.end(),
                     [&](int32_t a, int32_t b) { return B->n_layers[a] > B->n_layers[b]; });
    auto anchor = [&](int32_t m, int32_t j) {
        return (j - B->woff[m]) % SEARCH_STRIDE == 0 || j == B->woff[m + 1] - 1;
    };
    B->search_order.reserve(nw);
    for (int32_t m : by_layers)
        for (int32_t j = B->woff[m]; j < B->woff[m + 1]; ++j)
            if (anchor(m, j)) B->search_order.push_back(j);
    B->n_anchor = (int32_t)B->search_order.size();
    for (int32_t m : by_layers)
        for (int32_t j = B->woff[m]; j < B->woff[m + 1]; ++j)
            if (!anchor(m, j)) B->search_order.push_back(j);
    // The certificate's order: model by model, the fewest layers first
    // (measured a little faster there than the other way round, beside the
    // second stream's chain). Left out when the models come in that order
    // already.
    if (!std::is_sorted(B->n_layers.begin(), B->n_layers.end())) {
        B->layer_order.reserve(nw);
        std::stable_sort(by_layers.begin(), by_layers.end(),
                         [&](int32_t a, int32_t b) { return B->n_layers[a] < B->n_layers[b]; });
        for (int32_t m : by_layers)
            for (int32_t j = B->woff[m]; j < B->woff[m + 1]; ++j) B->layer_order.push_back(j);
    }
    B->order_sorted = B->order_natural;
    std::stable_sort(B->order_sorted.begin(), B->order_sorted.end(),
                     [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    std::vector<double> rec;
    build_records(B, h, a, b, r, rec);
    std::vector<float> rec32;
    build_records32(B, rec, rec32);
    std::vector<float> recdf((size_t)B->n_records * LAYER_STRIDE_DF);
    for (int64_t i = 0; i < B->n_records; ++i)
        df_record(&rec[(size_t)i * LAYER_STRIDE], &recdf[(size_t)i * LAYER_STRIDE_DF]);

    if ((rc = masw_sm_count(&B->sm_count))) {
        free_batch(B);
        return rc;
    }
    if (dev_alloc(&B->d_layers, rec.size()) || dev_alloc(&B->d_loff, B->n_models + 1) ||
        dev_alloc(&B->d_woff, B->n_models + 1) || dev_alloc(&B->d_nlim, B->n_models) ||
        dev_alloc(&B->d_k, nw) || dev_alloc(&B->d_item_model, nw) ||
        dev_alloc(&B->d_order_sorted, nw) || dev_alloc(&B->d_order_natural, nw) ||
        dev_alloc(&B->d_search_order, nw) ||
        (!B->layer_order.empty() && dev_alloc(&B->d_layer_order, nw)) ||
        dev_alloc(&B->d_grad_off, nw + 1) || dev_alloc(&B->d_counter, 1) ||
        dev_alloc(&B->d_ct, nw) || dev_alloc(&B->d_idx, nw) || dev_alloc(&B->d_status, nw) ||
        dev_alloc(&B->d_layers32, rec32.size()) || dev_alloc(&B->d_layers_df, recdf.size()) ||
        dev_alloc(&B->d_n32, nw) || dev_alloc(&B->d_cert, nw) ||
        dev_alloc(&B->d_search, nw) || dev_alloc(&B->d_unres, nw) || dev_alloc(&B->d_fallback, nw) ||
        dev_alloc(&B->d_counters, 2 * SCAN_COUNTERS) || dev_alloc(&B->d_nsearch, nw) ||
        dev_alloc(&B->d_search2, nw) || dev_alloc(&B->d_unres2, nw) ||
        dev_alloc(&B->d_fallback2, nw)) {
        free_batch(B);
        return MASW_ENOMEM;
    }
    auto up = [&](void* d, const void* s, size_t bytes) {
        return bytes ? cudaMemcpy(d, s, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = up(B->d_layers, rec.data(), rec.size() * sizeof(double));
    if (e == cudaSuccess) e = up(B->d_layers32, rec32.data(), rec32.size() * sizeof(float));
    if (e == cudaSuccess) e = up(B->d_layers_df, recdf.data(), recdf.size() * sizeof(float));
    if (e == cudaSuccess) e = up(B->d_loff, B->loff.data(), B->loff.size() * 4);
    if (e == cudaSuccess) e = up(B->d_woff, B->woff.data(), B->woff.size() * 4);
    if (e == cudaSuccess) e = up(B->d_nlim, B->nlim.data(), B->nlim.size() * 4);
    if (e == cudaSuccess) e = up(B->d_k, B->kvec.data(), nw * 8);
    if (e == cudaSuccess) e = up(B->d_item_model, B->item_model.data(), nw * 4);
    if (e == cudaSuccess) e = up(B->d_order_sorted, B->order_sorted.data(), nw * 4);
    if (e == cudaSuccess) e = up(B->d_order_natural, B->order_natural.data(), nw * 4);
    if (e == cudaSuccess) e = up(B->d_search_order, B->search_order.data(), nw * 4);
    if (e == cudaSuccess && B->d_layer_order)
        e = up(B->d_layer_order, B->layer_order.data(), nw * 4);
    if (e == cudaSuccess) e = up(B->d_grad_off, B->grad_off.data(), (nw + 1) * 8);
    if (e == cudaSuccess) e = cudaEventCreate(&B->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&B->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&B->phase_ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&B->phase_ev[1]);
    if (e == cudaSuccess) e = cudaEventCreate(&B->phase_ev[2]);
    if (e == cudaSuccess) e = cudaEventCreate(&B->side_fork);
    if (e == cudaSuccess) e = cudaEventCreate(&B->side_join);
    if (e == cudaSuccess) {
        // the side stream at the device's highest priority, so that its few
        // blocks are dispatched ahead of the certificate's queued ones
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) {
            B->side_prio = greatest;
            e = cudaStreamCreateWithPriority(&B->side, cudaStreamNonBlocking, greatest);
        }
    }
    if (e != cudaSuccess) {
        record_cuda_error(e, "batch upload", __LINE__);
        free_batch(B);
        return MASW_ECUDA;
    }
    B->plan = default_plan(B);
    if ((rc = rebuild_graph(B))) {
        free_batch(B);
        return rc;
    }
    *out = B;
    return MASW_OK;
}

int masw_model_batch_destroy(masw_batch* B) {
    if (!B) return MASW_EINVAL;
    cudaStreamSynchronize(B->stream);
    free_batch(B);
    return MASW_OK;
}

int masw_model_batch_update(masw_batch* B, const double* h, const double* alpha, const double* beta,
                            const double* rho, int32_t mem_space) {
    if (!B || (mem_space != MASW_HOST && mem_space != MASW_DEVICE)) return MASW_EINVAL;
    const int64_t nh = B->n_records - B->n_models, nr = B->n_records;
    if ((nh > 0 && !h) || (nr > 0 && (!alpha || !beta || !rho))) return MASW_EINVAL;
    // staging for host arrays (h, alpha, beta, rho) and the validation flag
    if (!B->d_upd && dev_alloc(&B->d_upd, (size_t)(nh + 3 * nr))) return MASW_ENOMEM;
    if (!B->d_upd_err && dev_alloc(&B->d_upd_err, 1)) return MASW_ENOMEM;
    const double *dh = h, *da = alpha, *db = beta, *dr = rho;
    if (mem_space == MASW_HOST) {
        // host arrays: checked here with the creation rules, so the update is
        // queued without a round trip (the device check below then finds
        // nothing); the copies read the arrays when the stream reaches them
        if (validate_layers(B->n_layers.data(), B->n_layers.size(), h, alpha, beta, rho))
            return MASW_EINVAL;
        double* st = B->d_upd;
        dh = st;
        da = st + nh;
        db = st + nh + nr;
        dr = st + nh + 2 * nr;
        const double* src[4] = {h, alpha, beta, rho};
        double* dst[4] = {st, st + nh, st + nh + nr, st + nh + 2 * nr};
        const int64_t cnt[4] = {nh, nr, nr, nr};
        for (int q = 0; q < 4; ++q)
            if (cnt[q] > 0)
                CK(cudaMemcpyAsync(dst[q], src[q], cnt[q] * sizeof(double), cudaMemcpyHostToDevice,
                                   B->stream));
    }
    // queued after the work already on the batch stream: validation, then the
    // records and scan limits (skipped on a validation error), then the flag
    CK(cudaMemsetAsync(B->d_upd_err, 0, sizeof(int32_t), B->stream));
    CK(launch_model_update(B->dev(false), dh, da, db, dr, B->d_layers, B->d_layers32,
                           B->d_layers_df, B->d_nlim,
                           B->d_upd_err, B->stream));
    if (mem_space == MASW_HOST) return MASW_OK;
    // device arrays: one synchronisation returns the device check's flag
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, B->d_upd_err, sizeof(int32_t), cudaMemcpyDeviceToHost, B->stream));
    CK(cudaStreamSynchronize(B->stream));
    return err ? MASW_EINVAL : MASW_OK;
}

int masw_model_batch_update_beta_h(masw_batch* B, const double* h, const double* beta) {
    if (!B || !beta || (B->n_records > B->n_models && !h)) return MASW_EINVAL;
    int rc;
    double *dh = nullptr, *db = nullptr;
    int64_t nh = B->n_records - B->n_models;
    bool hdev = h ? is_device_ptr(h) : true, bdev = is_device_ptr(beta);
    if (!hdev || !bdev) {  // stage host arrays in the (lazily allocated) gradient buffers
        if ((rc = ensure(&B->d_gb, B->n_records)) || (rc = ensure(&B->d_gh, nh))) return rc;
        if ((rc = copy_in(B->d_gb, beta, B->n_records, B->stream))) return rc;
        if (nh && (rc = copy_in(B->d_gh, h, nh, B->stream))) return rc;
        db = B->d_gb;
        dh = B->d_gh;
    }
    if (bdev) db = const_cast<double*>(beta);
    if (hdev) dh = const_cast<double*>(h);
    int32_t herr = 0;
    CK(cudaMemsetAsync(B->d_counter, 0, sizeof(int32_t), B->stream));
    CK(launch_update_beta_h(B->dev(false), dh, db, B->d_layers, B->d_layers32, B->d_layers_df,
                            B->d_nlim,
                            B->d_counter, B->stream));
    CK(cudaMemcpyAsync(&herr, B->d_counter, sizeof(int32_t), cudaMemcpyDeviceToHost, B->stream));
    CK(cudaStreamSynchronize(B->stream));
    return herr ? MASW_EINVAL : MASW_OK;
}

int masw_batch_info(const masw_batch* B, int64_t* n_items, int32_t* n_models, int32_t* max_layers) {
    if (!B) return MASW_EINVAL;
    if (n_items) *n_items = B->n_items;
    if (n_models) *n_models = B->n_models;
    if (max_layers) *max_layers = B->max_layers;
    return MASW_OK;
}

static int finish_outputs(masw_batch* B, double* ct, int32_t* idx, int32_t* status) {
    bool sync = false;
    int rc;
    if ((rc = copy_out(ct, B->d_ct, B->n_items, B->stream, &sync)) ||
        (rc = copy_out(idx, B->d_idx, B->n_items, B->stream, &sync)) ||
        (rc = copy_out(status, B->d_status, B->n_items, B->stream, &sync)))
        return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_dispersion(masw_batch* B, double* ct, int32_t* ct_idx, int32_t* status,
                    int32_t out_mem_space) {
    if (!B || (out_mem_space != MASW_HOST && out_mem_space != MASW_DEVICE)) return MASW_EINVAL;
    int rc = run_scan(B);
    if (rc) return rc;
    return finish_outputs(B, ct, ct_idx, status);
}

int masw_dispersion_changes(masw_batch* B, int32_t max_changes, double* ct, int32_t* ct_idx,
                            int32_t* status, int32_t* delta_count, int32_t out_mem_space) {
    if (!B || max_changes < 1 || max_changes > MASW_MAX_CHANGES ||
        (out_mem_space != MASW_HOST && out_mem_space != MASW_DEVICE))
        return MASW_EINVAL;
    const size_t nw = B->n_items, ne = nw * (size_t)max_changes;
    if (max_changes > B->chg_cap) {
        void* old[] = {B->d_chg_ct, B->d_chg_idx, B->d_chg_status, B->d_chg_delta};
        for (void* q : old)
            if (q) cudaFree(q);
        B->d_chg_ct = nullptr;
        B->d_chg_idx = B->d_chg_status = B->d_chg_delta = nullptr;
        B->chg_cap = 0;
        if (dev_alloc(&B->d_chg_ct, ne) || dev_alloc(&B->d_chg_idx, ne) ||
            dev_alloc(&B->d_chg_status, ne) || dev_alloc(&B->d_chg_delta, ne))
            return MASW_ENOMEM;
        B->chg_cap = max_changes;
    }
    if (!B->d_chg_counters && dev_alloc(&B->d_chg_counters, CHANGES_COUNTERS + nw))
        return MASW_ENOMEM;
    // the first change: Algorithm 1 with the batch plan (an FP64 decision)
    int rc0 = run_scan(B);
    if (rc0) return rc0;
    CK(launch_changes(B->dev(B->plan.ordered != 0), to_scan_plan(B, B->plan), max_changes,
                      B->d_idx, B->plan.precision == 2 ? B->d_cert : nullptr, B->d_layers32,
                      B->d_chg_ct, B->d_chg_idx, B->d_chg_status, B->d_chg_delta,
                      B->d_chg_counters, B->d_chg_counters + CHANGES_COUNTERS,
                      B->plan.precision >= 1, B->stream));
    B->changes_counted = B->plan.precision >= 1;
    bool sync = false;
    int rc;
    if ((rc = copy_out(ct, B->d_chg_ct, ne, B->stream, &sync)) ||
        (rc = copy_out(ct_idx, B->d_chg_idx, ne, B->stream, &sync)) ||
        (rc = copy_out(status, B->d_chg_status, ne, B->stream, &sync)) ||
        (rc = copy_out(delta_count, B->d_chg_delta, ne, B->stream, &sync)))
        return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_dispersion_leaky(masw_batch* B, double* ct, int32_t* ct_idx, int32_t* status,
                          int32_t out_mem_space) {
    if (!B || (out_mem_space != MASW_HOST && out_mem_space != MASW_DEVICE)) return MASW_EINVAL;
    const size_t nw = B->n_items;
    if ((!B->d_lk_ct && dev_alloc(&B->d_lk_ct, std::max<size_t>(nw, 1))) ||
        (!B->d_lk_idx && dev_alloc(&B->d_lk_idx, 4 * nw + 4)))
        return MASW_ENOMEM;
    // below the half-space shear speed: Algorithm 1 with the batch plan
    int rc0 = run_scan(B);
    if (rc0) return rc0;
    int32_t* lk_status = B->d_lk_idx + nw;
    ScanOut o{B->d_lk_ct, B->d_lk_idx, lk_status};
    CK(launch_leaky(B->dev(B->plan.ordered != 0), to_scan_plan(B, B->plan), B->d_idx,
                    B->d_status, o, B->d_lk_idx + 2 * nw, B->plan.precision >= 1 ? 1 : 0,
                    B->stream));
    bool sync = false;
    int rc;
    if ((rc = copy_out(ct, B->d_lk_ct, nw, B->stream, &sync)) ||
        (rc = copy_out(ct_idx, B->d_lk_idx, nw, B->stream, &sync)) ||
        (rc = copy_out(status, lk_status, nw, B->stream, &sync)))
        return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_element_check(masw_batch* B, int32_t n, const int32_t* item, const int32_t* layer,
                       const double* c, int32_t dd_trig, double* fp64, double* df) {
    if (!B || n < 0 || (n > 0 && (!item || !layer || !c || !fp64 || !df))) return MASW_EINVAL;
    if (dd_trig != 0 && dd_trig != 1) return MASW_EINVAL;
    for (int32_t t = 0; t < n; ++t) {
        if (item[t] < 0 || item[t] >= B->n_items) return MASW_EINVAL;
        const int32_t m = B->item_model[item[t]];
        if (layer[t] < 0 || layer[t] >= B->n_layers[m] || !(std::isfinite(c[t]) && c[t] > 0.0))
            return MASW_EINVAL;
    }
    if (n == 0) return MASW_OK;
    // one buffer: item, layer (int32 each), c, then the two outputs (7 doubles per point)
    double* d = nullptr;
    if (dev_alloc(&d, (size_t)n * 16)) return MASW_ENOMEM;
    int32_t* d_item = reinterpret_cast<int32_t*>(d);
    int32_t* d_layer = d_item + n;
    double* d_c = d + n;
    double* d_fp = d_c + n;
    double* d_df = d_fp + 7 * (size_t)n;
    cudaStream_t s = B->stream;
    cudaError_t e = cudaMemcpyAsync(d_item, item, n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_layer, layer, n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_c, c, n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_element_check(B->dev(false), n, d_item, d_layer, d_c, dd_trig, d_fp, d_df, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(fp64, d_fp, 7 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(df, d_df, 7 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    CK(e);
    return MASW_OK;
}

int masw_sincos_check(int32_t n, const double* x, double* s_lib, double* c_lib, double* s_cuda,
                      double* c_cuda, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!x || !s_lib || !c_lib || !s_cuda || !c_cuda))) return MASW_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (!(x[i] >= 0.0 && x[i] <= 1.25 * 3.141592653589793)) return MASW_EINVAL;
    if (n == 0) return MASW_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* d = nullptr;
    if (dev_alloc(&d, 5 * (size_t)n)) return MASW_ENOMEM;
    const size_t nn = (size_t)n;
    cudaError_t e = cudaMemcpyAsync(d, x, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_sincos_check(n, d, d + nn, d + 2 * nn, d + 3 * nn, d + 4 * nn, s);
    double* outs[4] = {s_lib, c_lib, s_cuda, c_cuda};
    for (int q = 0; q < 4 && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(outs[q], d + (q + 1) * nn, nn * sizeof(double), cudaMemcpyDeviceToHost,
                            s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    CK(e);
    return MASW_OK;
}

int masw_exp_check(int32_t n, const double* x, double* y_lib, double* y_cuda, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!x || !y_lib || !y_cuda))) return MASW_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (!(x[i] <= 0.0)) return MASW_EINVAL;
    if (n == 0) return MASW_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* d = nullptr;
    if (dev_alloc(&d, 3 * (size_t)n)) return MASW_ENOMEM;
    cudaError_t e = cudaMemcpyAsync(d, x, n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_exp_check(n, d, d + n, d + 2 * (size_t)n, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_lib, d + n, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_cuda, d + 2 * (size_t)n, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    CK(e);
    return MASW_OK;
}

int masw_dispersion_plain(masw_batch* B, double* ct, int32_t* ct_idx, int32_t* status,
                          int32_t out_mem_space) {
    if (!B || (out_mem_space != MASW_HOST && out_mem_space != MASW_DEVICE)) return MASW_EINVAL;
    masw_plan p = B->plan;
    p.persistent = 0;
    p.ordered = 0;
    ScanOut o{B->d_ct, B->d_idx, B->d_status, B->d_cert};
    DevBatch d = B->dev(false);
    ScanPlan sp = to_scan_plan(B, p);
    B->phases_valid = false;  // the per-model launches record no phase events
    B->count_phases_valid = false;
    B->side_phase_valid = false;
    CK(cudaEventRecord(B->ev0, B->stream));
    for (int32_t m = 0; m < B->n_models; ++m) {
        if (p.precision >= 1)
            CK(launch_screen_scan(d, o, sp, B->d_layers32, B->d_n32, B->d_search, B->d_unres,
                                  B->d_fallback, B->d_counters, p.precision == 2, B->woff[m],
                                  B->woff[m + 1], B->stream, nullptr, nullptr));
        else
            CK(launch_scan(d, o, sp, B->d_counter, B->woff[m], B->woff[m + 1], B->stream));
        CK(cudaStreamSynchronize(B->stream));
    }
    CK(cudaEventRecord(B->ev1, B->stream));
    return finish_outputs(B, ct, ct_idx, status);
}

int masw_last_scan_phases(const masw_batch* B, float* ms) {
    if (!B || !ms) return MASW_EINVAL;
    if (!B->phases_valid) return MASW_EINVAL;
    CK(cudaEventSynchronize(B->ev1));
    CK(cudaEventElapsedTime(&ms[0], B->ev0, B->phase_ev[0]));
    CK(cudaEventElapsedTime(&ms[1], B->phase_ev[0], B->phase_ev[1]));
    CK(cudaEventElapsedTime(&ms[2], B->phase_ev[1], B->ev1));
    return MASW_OK;
}

int masw_last_count_phases(const masw_batch* B, float* ms) {
    if (!B || !ms) return MASW_EINVAL;
    if (!B->count_phases_valid) return MASW_EINVAL;
    CK(cudaEventSynchronize(B->ev1));
    CK(cudaEventElapsedTime(&ms[0], B->ev0, B->phase_ev[2]));
    CK(cudaEventElapsedTime(&ms[1], B->phase_ev[2], B->phase_ev[0]));
    ms[2] = 0.f;
    if (B->side_phase_valid) CK(cudaEventElapsedTime(&ms[2], B->side_fork, B->side_join));
    return MASW_OK;
}

int masw_last_scan_screen(masw_batch* B, int32_t* n32) {
    if (!B || !n32 || B->plan.precision < 1) return MASW_EINVAL;
    bool sync = false;
    int rc = copy_out(n32, B->d_n32, B->n_items, B->stream, &sync);
    if (rc) return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_last_scan_unresolved(const masw_batch* B, int32_t* n) {
    if (!B || !n) return MASW_EINVAL;
    if (B->plan.precision < 1) {
        *n = -1;
        return MASW_OK;
    }
    int32_t v[2 * SCAN_COUNTERS];
    CK(cudaStreamSynchronize(B->stream));
    CK(cudaMemcpy(v, B->d_counters, sizeof(v), cudaMemcpyDeviceToHost));
    *n = v[5] + v[SCAN_COUNTERS + 5];
    return MASW_OK;
}

int masw_last_scan_fallback(const masw_batch* B, int32_t* n) {
    if (!B || !n) return MASW_EINVAL;
    if (B->plan.precision != 2) {
        *n = -1;
        return MASW_OK;
    }
    int32_t v[2 * SCAN_COUNTERS];
    CK(cudaStreamSynchronize(B->stream));
    CK(cudaMemcpy(v, B->d_counters, sizeof(v), cudaMemcpyDeviceToHost));
    *n = v[3] + v[SCAN_COUNTERS + 3];
    return MASW_OK;
}

int masw_last_changes_linear(const masw_batch* B, int32_t* n) {
    if (!B || !n) return MASW_EINVAL;
    if (!B->changes_counted || !B->d_chg_counters) {
        *n = -1;
        return MASW_OK;
    }
    int32_t v = 0;
    CK(cudaStreamSynchronize(B->stream));
    CK(cudaMemcpy(&v, B->d_chg_counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost));
    *n = v;
    return MASW_OK;
}

int masw_last_scan_ms(const masw_batch* B, float* ms) {
    if (!B || !ms) return MASW_EINVAL;
    CK(cudaEventSynchronize(B->ev1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, B->ev0, B->ev1));
    *ms = t;
    return MASW_OK;
}

int masw_misfit(masw_batch* B, const double* ce, int32_t kind, double sigma, double* misfit) {
    if (!B || !ce || !misfit || (kind != MASW_MISFIT_PAPER && kind != MASW_MISFIT_LSQ))
        return MASW_EINVAL;
    if (kind == MASW_MISFIT_LSQ && !(sigma > 0.0 && std::isfinite(sigma))) return MASW_EINVAL;
    int rc;
    if ((rc = ensure(&B->d_ce, B->n_items)) || (rc = ensure(&B->d_misfit, B->n_models))) return rc;
    if ((rc = copy_in(B->d_ce, ce, B->n_items, B->stream))) return rc;
    if ((rc = run_scan(B))) return rc;
    CK(launch_misfit(B->dev(false), B->d_ct, B->d_ce, kind, sigma, B->d_misfit, nullptr, B->stream));
    bool sync = false;
    if ((rc = copy_out(misfit, B->d_misfit, B->n_models, B->stream, &sync))) return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_misfit_curves(masw_batch* B, const double* ce, int32_t kind, double sigma,
                       double* misfit, double* ct, int32_t* ct_idx, int32_t* status) {
    if (!B || !ce || !misfit || (kind != MASW_MISFIT_PAPER && kind != MASW_MISFIT_LSQ))
        return MASW_EINVAL;
    if (kind == MASW_MISFIT_LSQ && !(sigma > 0.0 && std::isfinite(sigma))) return MASW_EINVAL;
    int rc;
    if ((rc = ensure(&B->d_ce, B->n_items)) || (rc = ensure(&B->d_misfit, B->n_models))) return rc;
    // the observed curve goes in without a wait: the one synchronisation at
    // the end covers the caller's host buffer as well
    bool sync = !is_device_ptr(ce);
    if (B->n_items > 0)
        CK(cudaMemcpyAsync(B->d_ce, ce, B->n_items * sizeof(double),
                           sync ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, B->stream));
    if ((rc = run_scan(B))) return rc;
    CK(launch_misfit(B->dev(false), B->d_ct, B->d_ce, kind, sigma, B->d_misfit, nullptr, B->stream));
    if ((rc = copy_out(misfit, B->d_misfit, B->n_models, B->stream, &sync)) ||
        (rc = copy_out(ct, B->d_ct, B->n_items, B->stream, &sync)) ||
        (rc = copy_out(ct_idx, B->d_idx, B->n_items, B->stream, &sync)) ||
        (rc = copy_out(status, B->d_status, B->n_items, B->stream, &sync)))
        return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

static int run_roots(masw_batch* B) {
    int rc;
    if ((rc = ensure(&B->d_croot, B->n_items))) return rc;
    if ((rc = run_scan(B))) return rc;
    CK(launch_refine(B->dev(false), B->d_idx, 1e-13, B->d_croot, B->stream));
    return MASW_OK;
}

static int run_root_grad(masw_batch* B) {
    int rc;
    if ((rc = ensure(&B->d_rows, B->grad_len)) ||
        (rc = ensure(&B->d_bs, 12 * (B->grad_len + B->n_items))))
        return rc;
    if ((rc = run_roots(B))) return rc;
    CK(launch_root_grad(B->dev(false), B->d_croot, B->d_rows, B->d_bs, B->stream));
    return MASW_OK;
}

int masw_roots(masw_batch* B, double* croot) {
    if (!B || !croot) return MASW_EINVAL;
    int rc = run_roots(B);
    if (rc) return rc;
    bool sync = false;
    if ((rc = copy_out(croot, B->d_croot, B->n_items, B->stream, &sync))) return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_root_grad(masw_batch* B, double* rows, int64_t* row_len_total) {
    if (!B) return MASW_EINVAL;
    if (row_len_total) *row_len_total = B->grad_len;
    if (!rows) return MASW_OK;
    int rc = run_root_grad(B);
    if (rc) return rc;
    bool sync = false;
    if ((rc = copy_out(rows, B->d_rows, B->grad_len, B->stream, &sync))) return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_misfit_grad(masw_batch* B, const double* ce, int32_t kind, double sigma, double* misfit,
                     double* grad_beta, double* grad_h) {
    if (!B || !ce || !misfit || (kind != MASW_MISFIT_PAPER && kind != MASW_MISFIT_LSQ))
        return MASW_EINVAL;
    if (kind == MASW_MISFIT_LSQ && !(sigma > 0.0 && std::isfinite(sigma))) return MASW_EINVAL;
    int rc;
    if ((rc = ensure(&B->d_ce, B->n_items)) || (rc = ensure(&B->d_misfit, B->n_models)) ||
        (rc = ensure(&B->d_dphi, B->n_items)) || (rc = ensure(&B->d_gb, B->n_records)) ||
        (rc = ensure(&B->d_gh, B->n_records - B->n_models)))
        return rc;
    if ((rc = copy_in(B->d_ce, ce, B->n_items, B->stream))) return rc;
    if ((rc = run_root_grad(B))) return rc;
    DevBatch d = B->dev(false);
    CK(launch_misfit(d, B->d_croot, B->d_ce, kind, sigma, B->d_misfit, B->d_dphi, B->stream));
    CK(launch_grad_reduce(d, B->d_rows, B->d_dphi, B->d_gb, B->d_gh, B->stream));
    bool sync = false;
    if ((rc = copy_out(misfit, B->d_misfit, B->n_models, B->stream, &sync)) ||
        (rc = copy_out(grad_beta, B->d_gb, B->n_records, B->stream, &sync)) ||
        (rc = copy_out(grad_h, B->d_gh, B->n_records - B->n_models, B->stream, &sync)))
        return rc;
    if (sync) CK(cudaStreamSynchronize(B->stream));
    return MASW_OK;
}

int masw_det_eval(masw_batch* B, int32_t n, const int32_t* item, const double* c, int32_t* sign,
                  double* log_abs) {
    if (!B || n < 0 || (n > 0 && (!item || !c || !sign || !log_abs))) return MASW_EINVAL;
    if (n == 0) return MASW_OK;
    int32_t *d_item = nullptr, *d_sign = nullptr;
    double *d_c = nullptr, *d_la = nullptr;
    int rc = MASW_OK;
    if (dev_alloc(&d_item, n) || dev_alloc(&d_sign, n) || dev_alloc(&d_c, n) || dev_alloc(&d_la, n))
        rc = MASW_ENOMEM;
    bool sync = false;
    if (!rc) rc = copy_in(d_item, item, n, B->stream);
    if (!rc) rc = copy_in(d_c, c, n, B->stream);
    if (!rc) {
        cudaError_t e = launch_det_eval(B->dev(false), n, d_item, d_c, d_sign, d_la, B->stream);
        if (e != cudaSuccess) {
            record_cuda_error(e, "det_eval", __LINE__);
            rc = MASW_ECUDA;
        }
    }
    if (!rc) rc = copy_out(sign, d_sign, n, B->stream, &sync);
    if (!rc) rc = copy_out(log_abs, d_la, n, B->stream, &sync);
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (!rc && e != cudaSuccess) {
        record_cuda_error(e, "det_eval sync", __LINE__);
        rc = MASW_ECUDA;
    }
    cudaFree(d_item);
    cudaFree(d_sign);
    cudaFree(d_c);
    cudaFree(d_la);
    return rc;
}

int masw_mode_count(masw_batch* B, int32_t n, const int32_t* item, const double* c, int32_t* s,
                    int32_t* j0) {
    if (!B || n < 0 || (n > 0 && (!item || !c || !s || !j0))) return MASW_EINVAL;
    if (n == 0) return MASW_OK;
    int32_t *d_item = nullptr, *d_s = nullptr, *d_j0 = nullptr;
    double* d_c = nullptr;
    int rc = MASW_OK;
    if (dev_alloc(&d_item, n) || dev_alloc(&d_s, n) || dev_alloc(&d_j0, n) || dev_alloc(&d_c, n))
        rc = MASW_ENOMEM;
    bool sync = false;
    if (!rc) rc = copy_in(d_item, item, n, B->stream);
    if (!rc) rc = copy_in(d_c, c, n, B->stream);
    if (!rc) {
        cudaError_t e = launch_mode_count(B->dev(false), n, d_item, d_c, d_s, d_j0, B->stream);
        if (e != cudaSuccess) {
            record_cuda_error(e, "mode_count", __LINE__);
            rc = MASW_ECUDA;
        }
    }
    if (!rc) rc = copy_out(s, d_s, n, B->stream, &sync);
    if (!rc) rc = copy_out(j0, d_j0, n, B->stream, &sync);
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (!rc && e != cudaSuccess) {
        record_cuda_error(e, "mode_count sync", __LINE__);
        rc = MASW_ECUDA;
    }
    cudaFree(d_item);
    cudaFree(d_s);
    cudaFree(d_j0);
    cudaFree(d_c);
    return rc;
}

int masw_get_plan(const masw_batch* B, masw_plan* plan) {
    if (!B || !plan) return MASW_EINVAL;
    *plan = B->plan;
    return MASW_OK;
}

int masw_set_plan(masw_batch* B, const masw_plan* plan) {
    if (!B || !plan || !plan_ok(*plan)) return MASW_EINVAL;
    CK(cudaStreamSynchronize(B->stream));
    B->plan = *plan;
    return rebuild_graph(B);
}

int masw_test_fail_alloc(int32_t k) {
    g_alloc_fail_at.store(k < 0 ? -1 : (int)k);
    return MASW_OK;
}

int masw_set_route(masw_batch* B, int32_t route) {
    if (!B || route < 0 || route > 4) return MASW_EINVAL;
    CK(cudaStreamSynchronize(B->stream));
    B->route = route;
    return rebuild_graph(B);
}

// ----------------------------------------------------------- autotuner

namespace {
std::mutex g_cache_mu;
std::map<std::tuple<int, int, int>, masw_plan> g_cache;
bool g_cache_loaded = false;

std::tuple<int, int, int> cache_key(const masw_batch* B) {
    int bucket = 0;
    for (int64_t n = B->n_items; n > 1; n >>= 1) ++bucket;
    return {B->max_layers * 2 + B->plan.precision, B->grid.n_c, bucket};
}

void load_cache_file() {
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    const char* path = getenv("MASW_PLAN_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    int a, b, c;
    masw_plan p;
    while (fscanf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d", &a, &b, &c, &p.warps_per_block,
                  &p.cpl, &p.blocks_per_sm, &p.persistent, &p.ordered, &p.stage_layers,
                  &p.use_graph, &p.precision, &p.count_block, &p.count_split) == 13)
        if (plan_ok(p)) g_cache[{a, b, c}] = p;
    fclose(f);
}

void save_cache_file() {
    const char* path = getenv("MASW_PLAN_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (auto& kv : g_cache) {
        const masw_plan& p = kv.second;
        fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d %d\n", std::get<0>(kv.first),
                std::get<1>(kv.first), std::get<2>(kv.first), p.warps_per_block, p.cpl,
                p.blocks_per_sm, p.persistent, p.ordered, p.stage_layers, p.use_graph, p.precision,
                p.count_block, p.count_split);
    }
    fclose(f);
}
}  // namespace

int masw_autotune(masw_batch* B, int32_t reps, masw_plan* best) {
    if (!B || reps < 1) return MASW_EINVAL;
    auto key = cache_key(B);
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        load_cache_file();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            int rc = masw_set_plan(B, &it->second);
            if (rc) return rc;
            if (best) *best = it->second;
            return MASW_OK;
        }
    }
    // median of reps timed scans (one warm-up scan first) of a candidate
    auto time_plan = [&](const masw_plan& p, float* ms_out) -> int {
        int rc = masw_set_plan(B, &p);
        if (rc) return rc;
        if ((rc = run_scan(B))) return rc;  // warm-up
        std::vector<float> t;
        for (int r = 0; r < reps; ++r) {
            if ((rc = run_scan(B))) return rc;
            float ms;
            if ((rc = masw_last_scan_ms(B, &ms))) return rc;
            t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        *ms_out = t[t.size() / 2];
        return MASW_OK;
    };
    masw_plan bestp = B->plan;
    bestp.persistent = 1;
    bestp.use_graph = 1;
    bestp.stage_layers = std::min(B->max_layers + 1, 32);
    float best_ms = 1e30f;
    auto consider = [&](const masw_plan& p) -> int {
        if (!plan_ok(p)) return MASW_OK;
        float ms = 0.f;
        int rc = time_plan(p, &ms);
        if (rc) return rc;
        if (ms < best_ms) {
            best_ms = ms;
            bestp = p;
        }
        return MASW_OK;
    };
    int rc = consider(bestp);
    // stage 1: the counting kernel's block size (its launch bounds follow),
    // with the search in the same kernel or in one of its own
    if (!rc && bestp.precision == 2) {
        const masw_plan base = bestp;
        for (int split : {0, 1, 2}) {
            for (int cb : {64, 128, 256}) {
                masw_plan p = base;
                p.count_block = cb;
                p.count_split = split;
                if ((rc = consider(p))) break;
            }
            if (rc) break;
        }
    }
    // stage 2: warps per block x persistent blocks per SM of the other kernels
    if (!rc) {
        const masw_plan base = bestp;
        for (int wpb : {1, 2, 4, 8})
            for (int bps : {1, 2, 4, 8, 16}) {
                masw_plan p = base;
                p.warps_per_block = wpb;
                p.blocks_per_sm = bps;
                if ((rc = consider(p))) break;
            }
    }
    // stage 3: test velocities per lane x queue order
    if (!rc) {
        const masw_plan base = bestp;
        for (int cpl : {1, 2, 4})
            for (int ord : {0, 1}) {
                masw_plan p = base;
                p.cpl = cpl;
                p.ordered = ord;
                if ((rc = consider(p))) break;
            }
    }
    // last: one item per warp, no queue
    if (!rc) {
        masw_plan p = bestp;
        p.persistent = 0;
        rc = consider(p);
    }
    if (rc) return rc;
    rc = masw_set_plan(B, &bestp);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_cache[key] = bestp;
        save_cache_file();
    }
    if (best) *best = bestp;
    return MASW_OK;
}

int masw_fp64_peak(void* cuda_stream, double* flops) {
    if (!flops) return MASW_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int32_t sms = 0;
    int rc = masw_sm_count(&sms);
    if (rc) return rc;
    double* sink = nullptr;
    if (dev_alloc(&sink, 4096)) return MASW_ENOMEM;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    const int threads = 256, iters = 2048;
    const int blocks = sms * 8;
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(a, s));
        CK(launch_fp64_peak(blocks, threads, iters, sink, s));
        CK(cudaEventRecord(b, s));
        CK(cudaEventSynchronize(b));
        CK(cudaEventElapsedTime(&ms, a, b));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    double dfma = (double)blocks * threads * iters * 16.0 * 8.0;
    *flops = 2.0 * dfma / (ms * 1e-3);
    return MASW_OK;
}

}  // extern "C"
