// masw_noalloc.cu -- masw_dispersion_noalloc: Algorithm 1 for a ragged batch
// without any device or host allocation by the library.
//
// Some callers cannot allocate GPU memory on their own: code that runs
// under a framework's caching allocator or a fixed memory budget, real-time
// services that forbid allocation after start-up, and embedders that only
// hand out pre-allocated buffers. masw_model_batch_create does allocate
// (it owns a device copy of the batch). This entry point instead keeps
// everything it derives from the inputs -- layer records (FP64, FP32 and
// double-float), offsets, scan limits, wavenumbers, the item order, the
// counting search's per-item lists and their counters -- in one file-scope
// device array of fixed size, and writes the results straight into the
// caller's output buffers. It runs the batch path's default counting plan in
// its fused form (the form that plan takes for batches of this size).
//
// The array lives for the whole process on every device that loads the
// library. Host code must not hand its symbol to a kernel (on the host the
// name is only a stand-in); the device address comes from
// cudaGetSymbolAddress, taken once per device, with that device current, on
// the first call made there.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/masw.h"
#include "masw_device.cuh"
#include "masw_df.cuh"
#include "masw_internal.h"
#include "masw_screen.cuh"

using namespace masw;

namespace {

// Scratch layout (byte offsets inside the array; every region 256-aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_RECORDS = 0;
constexpr size_t SZ_RECORDS = (size_t)MASW_NOALLOC_MAX_RECORDS * LAYER_STRIDE * sizeof(double);
constexpr size_t OFF_K = align256(OFF_RECORDS + SZ_RECORDS);
constexpr size_t SZ_K = (size_t)MASW_NOALLOC_MAX_ITEMS * sizeof(double);
constexpr size_t OFF_ITEM_MODEL = align256(OFF_K + SZ_K);
constexpr size_t SZ_ITEMS_I32 = (size_t)MASW_NOALLOC_MAX_ITEMS * sizeof(int32_t);
constexpr size_t OFF_ORDER = align256(OFF_ITEM_MODEL + SZ_ITEMS_I32);
constexpr size_t OFF_LOFF = align256(OFF_ORDER + SZ_ITEMS_I32);
constexpr size_t SZ_MODELS1_I32 = ((size_t)MASW_NOALLOC_MAX_MODELS + 1) * sizeof(int32_t);
constexpr size_t OFF_WOFF = align256(OFF_LOFF + SZ_MODELS1_I32);
constexpr size_t OFF_NLIM = align256(OFF_WOFF + SZ_MODELS1_I32);
constexpr size_t OFF_STAGE = align256(OFF_NLIM + SZ_MODELS1_I32);  // host inputs: h, alpha, beta, rho
constexpr size_t SZ_STAGE_LAYERS = (size_t)MASW_NOALLOC_MAX_RECORDS * sizeof(double);
constexpr size_t OFF_STAGE_LAMBDA = align256(OFF_STAGE + 4 * SZ_STAGE_LAYERS);
constexpr size_t OFF_REC32 = align256(OFF_STAGE_LAMBDA + SZ_K);
constexpr size_t SZ_REC32 = (size_t)MASW_NOALLOC_MAX_RECORDS * LAYER_STRIDE32 * sizeof(float);
constexpr size_t OFF_RECDF = align256(OFF_REC32 + SZ_REC32);
constexpr size_t SZ_RECDF = (size_t)MASW_NOALLOC_MAX_RECORDS * LAYER_STRIDE_DF * sizeof(float);
constexpr size_t OFF_N32 = align256(OFF_RECDF + SZ_RECDF);  // then search, re-scan, fallback lists
constexpr size_t OFF_LISTS = align256(OFF_N32 + SZ_ITEMS_I32);
constexpr size_t OFF_SCAN_COUNTERS = align256(OFF_LISTS + 3 * SZ_ITEMS_I32);
constexpr size_t OFF_COUNTER = align256(OFF_SCAN_COUNTERS + 2 * SCAN_COUNTERS * sizeof(int32_t));
constexpr size_t OFF_ERROR = OFF_COUNTER + 64;
constexpr size_t SCRATCH_BYTES = align256(OFF_ERROR + 64);
static_assert(SCRATCH_BYTES == MASW_NOALLOC_SCRATCH_BYTES, "scratch size must match masw.h");

constexpr int MAX_DEVICES = 64;

}  // namespace

// The scratch itself: one array per device context, kept until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device (set-up once
// per device, with that device current).
int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MASW_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return MASW_EINVAL;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MASW_ECUDA;
        }
        g_scratch_ptr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_ptr[dev];
    return MASW_OK;
}

// Memory type of a pointer as the CUDA runtime sees it; pageable host memory
// the runtime has never seen reads as cudaMemoryTypeUnregistered.
cudaMemoryType memory_type(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return cudaMemoryTypeUnregistered;
    }
    return a.type;
}

bool is_device(const void* p) {
    const cudaMemoryType t = memory_type(p);
    return t == cudaMemoryTypeDevice || t == cudaMemoryTypeManaged;
}

// An input array the declared space can read: device (or managed) memory for
// MASW_DEVICE, anything but plain device memory for MASW_HOST. A host array
// passed as MASW_DEVICE would reach the prep kernel as an illegal address,
// and a device array passed as MASW_HOST would be read on the host.
bool in_space(const void* p, bool dev_in) {
    return dev_in ? is_device(p) : memory_type(p) != cudaMemoryTypeDevice;
}

__device__ __forceinline__ bool fpos(double x) { return isfinite(x) && x > 0.0; }

// Validate the model values and derive the layer records, wavenumbers, item
// model/order and per-model scan limits (the same quantities and the same
// arithmetic as masw_model_batch_create). One thread per record, per item
// and per model; any invalid value sets *err.
__global__ void noalloc_prep_kernel(int n_models, const int32_t* __restrict__ loff,
                                    const int32_t* __restrict__ woff, const double* __restrict__ h,
                                    const double* __restrict__ alpha, const double* __restrict__ beta,
                                    const double* __restrict__ rho, const double* __restrict__ lam,
                                    masw_grid grid, double* records, float* records32,
                                    float* records_df, double* kvec, int32_t* item_model,
                                    int32_t* order, int32_t* nlim, int32_t* counter,
                                    int32_t* err) {
    const int n_rec = loff[n_models];
    const int n_items = woff[n_models];
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) *counter = 0;
    for (int m = t0; m < n_models; m += stride) {
        int N = loff[m + 1] - loff[m] - 1;
        int rec0 = loff[m];
        int h0 = rec0 - m;  // finite-layer offset: sum of N over earlier models
        for (int i = 0; i <= N; ++i) {
            int il = rec0 + i;
            double a = alpha[il], b = beta[il], r = rho[il];
            double hh = (i < N) ? h[h0 + i] : 0.0;
            bool ok = fpos(a) && fpos(b) && fpos(r) && (3.0 * a * a > 4.0 * b * b) &&
                      (i == N || fpos(hh));
            if (!ok) atomicOr(err, 1);
            double* L = records + (size_t)il * LAYER_STRIDE;
            L[L_H] = hh;
            L[L_MU] = r * b * b;
            L[L_RHO] = r;
            L[L_IA2] = 1.0 / (a * a);
            L[L_IB2] = 1.0 / (b * b);
            L[L_BETA] = b;
            L[L_RATIO] = a / b;
            L[L_IRHO] = 1.0 / r;
        }
        // the FP32 records of the search (stiffnesses over the half-space's
        // shear modulus) and the certificate's double-float records
        const double mref = records[(size_t)(rec0 + N) * LAYER_STRIDE + L_MU];
        for (int i = 0; i <= N; ++i) {
            const double* L = records + (size_t)(rec0 + i) * LAYER_STRIDE;
            float* F = records32 + (size_t)(rec0 + i) * LAYER_STRIDE32;
            for (int q = 0; q < LAYER_STRIDE32; ++q) F[q] = 0.0f;
            F[F_H] = (float)L[L_H];
            F[F_MU] = (float)(L[L_MU] / mref);
            F[F_RHO] = (float)(L[L_RHO] / mref);
            F[F_IA2] = (float)L[L_IA2];
            F[F_IB2] = (float)L[L_IB2];
            F[F_DIB] = (float)(L[L_IB2] - L[L_IA2]);
            df_record(L, records_df + (size_t)(rec0 + i) * LAYER_STRIDE_DF);
        }
        // grid points with V[n] < beta of the half-space
        double bhs = beta[rec0 + N];
        double est = floor((bhs - grid.c0) / grid.dc);
        long long n = (long long)fmax(0.0, fmin(est, (double)grid.n_c));
        while (n > 0 && !(grid_c(grid.c0, grid.dc, (int)(n - 1)) < bhs)) --n;
        while (n < grid.n_c && grid_c(grid.c0, grid.dc, (int)n) < bhs) ++n;
        nlim[m] = (int32_t)n;
        for (int j = woff[m]; j < woff[m + 1]; ++j) {
            double l = lam[j];
            if (!fpos(l)) atomicOr(err, 1);
            kvec[j] = 2.0 * M_PI / l;
            item_model[j] = m;
            order[j] = j;
        }
    }
    (void)n_rec;
    (void)n_items;
}

}  // namespace

extern "C" int masw_dispersion_noalloc(const masw_models_desc* md, const masw_grid* grid,
                                       void* cuda_stream, double* ct, int32_t* ct_idx,
                                       int32_t* status) {
    if (!md || !grid || !ct || !ct_idx || !status) return MASW_EINVAL;
    if (md->mem_space != MASW_HOST && md->mem_space != MASW_DEVICE) return MASW_EINVAL;
    if (md->n_models < 1) return MASW_EINVAL;
    if (md->n_models > MASW_NOALLOC_MAX_MODELS) return MASW_ETOOBIG;
    if (!(std::isfinite(grid->c0) && grid->c0 > 0.0 && std::isfinite(grid->dc) && grid->dc > 0.0 &&
          grid->n_c >= 2))
        return MASW_EINVAL;
    if (!md->n_layers || !md->n_lambda || !md->alpha || !md->beta || !md->rho || !md->lambda)
        return MASW_EINVAL;
    if (!is_device(ct) || !is_device(ct_idx) || !is_device(status)) return MASW_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool dev_in = md->mem_space == MASW_DEVICE;
    // every input array in the declared space, before any copy or launch
    const void* inputs[] = {md->n_layers, md->n_lambda, md->h, md->alpha, md->beta, md->rho,
                            md->lambda};
    for (const void* in : inputs)
        if (in && !in_space(in, dev_in)) return MASW_EINVAL;
    const int M = md->n_models;

    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;

    // model sizes and offsets on the host stack
    int32_t nl[MASW_NOALLOC_MAX_MODELS], nw[MASW_NOALLOC_MAX_MODELS];
    int32_t loff[MASW_NOALLOC_MAX_MODELS + 1], woff[MASW_NOALLOC_MAX_MODELS + 1];
    if (dev_in) {
        if (cudaMemcpy(nl, md->n_layers, M * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(nw, md->n_lambda, M * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return MASW_ECUDA;
        }
    } else {
        std::memcpy(nl, md->n_layers, M * sizeof(int32_t));
        std::memcpy(nw, md->n_lambda, M * sizeof(int32_t));
    }
    int64_t rec = 0, items = 0;
    int max_n = 0;
    loff[0] = woff[0] = 0;
    for (int m = 0; m < M; ++m) {
        if (nl[m] < 0 || nl[m] > MASW_MAX_LAYERS || nw[m] < 0) return MASW_EINVAL;
        rec += nl[m] + 1;
        items += nw[m];
        if (rec > MASW_NOALLOC_MAX_RECORDS || items > MASW_NOALLOC_MAX_ITEMS) return MASW_ETOOBIG;
        loff[m + 1] = (int32_t)rec;
        woff[m + 1] = (int32_t)items;
        max_n = nl[m] > max_n ? nl[m] : max_n;
    }
    if (rec - M > 0 && !md->h) return MASW_EINVAL;

    double* records = (double*)(base + OFF_RECORDS);
    float* records32 = (float*)(base + OFF_REC32);
    float* records_df = (float*)(base + OFF_RECDF);
    int32_t* n32 = (int32_t*)(base + OFF_N32);
    int32_t* lists = (int32_t*)(base + OFF_LISTS);
    int32_t* scan_counters = (int32_t*)(base + OFF_SCAN_COUNTERS);
    double* kvec = (double*)(base + OFF_K);
    int32_t* item_model = (int32_t*)(base + OFF_ITEM_MODEL);
    int32_t* order = (int32_t*)(base + OFF_ORDER);
    int32_t* d_loff = (int32_t*)(base + OFF_LOFF);
    int32_t* d_woff = (int32_t*)(base + OFF_WOFF);
    int32_t* d_nlim = (int32_t*)(base + OFF_NLIM);
    int32_t* counter = (int32_t*)(base + OFF_COUNTER);
    int32_t* err = (int32_t*)(base + OFF_ERROR);

    const double *h = md->h, *a = md->alpha, *b = md->beta, *r = md->rho, *lam = md->lambda;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, kind, s);
    };
    cp(d_loff, loff, (M + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    cp(d_woff, woff, (M + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (!dev_in) {  // stage host inputs in the scratch
        double* st = (double*)(base + OFF_STAGE);
        double* sh = st;
        double* sa = st + MASW_NOALLOC_MAX_RECORDS;
        double* sb = st + 2 * MASW_NOALLOC_MAX_RECORDS;
        double* sr = st + 3 * MASW_NOALLOC_MAX_RECORDS;
        double* sl = (double*)(base + OFF_STAGE_LAMBDA);
        cp(sh, h, (rec - M) * sizeof(double), cudaMemcpyHostToDevice);
        cp(sa, a, rec * sizeof(double), cudaMemcpyHostToDevice);
        cp(sb, b, rec * sizeof(double), cudaMemcpyHostToDevice);
        cp(sr, r, rec * sizeof(double), cudaMemcpyHostToDevice);
        cp(sl, lam, items * sizeof(double), cudaMemcpyHostToDevice);
        h = sh; a = sa; b = sb; r = sr; lam = sl;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) {
        int threads = 128;
        int blocks = (M + threads - 1) / threads;
        noalloc_prep_kernel<<<blocks, threads, 0, s>>>(M, d_loff, d_woff, h, a, b, r, lam, *grid,
                                                       records, records32, records_df, kvec,
                                                       item_model, order, d_nlim, counter, err);
        e = cudaGetLastError();
    }
    int32_t herr = 0;
    // the stack copies above must land before this frame returns; the error
    // word decides whether the scan runs
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MASW_ECUDA;
    }
    if (herr) return MASW_EINVAL;
    if (items == 0) return MASW_OK;

    int sms = 0, devn = 0;
    if (cudaGetDevice(&devn) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devn) != cudaSuccess) {
        cudaGetLastError();
        return MASW_ECUDA;
    }
    DevBatch d;
    d.layers = records;
    d.layers_df = records_df;
    d.model_loff = d_loff;
    d.model_nlim = d_nlim;
    d.model_woff = d_woff;
    d.k = kvec;
    d.item_model = item_model;
    d.order = order;
    d.grad_off = nullptr;
    d.n_models = M;
    d.n_items = (int32_t)items;
    d.c0 = grid->c0;
    d.dc = grid->dc;
    d.n_c = grid->n_c;
    d.route = 0;
    // the counting plan's fused form: search and certificate in one kernel,
    // then the fallback chain over the lists in the scratch
    ScanPlan p;
    p.warps_per_block = 8;
    p.cpl = 2;
    p.blocks = 4 * sms;
    p.persistent = 1;
    p.stage_layers = max_n + 1 < 32 ? max_n + 1 : 32;
    p.count_block = 128;
    p.count_split = 0;
    p.sms = sms;
    ScanOut o{ct, ct_idx, status};
    e = launch_screen_scan(d, o, p, records32, n32, lists, lists + MASW_NOALLOC_MAX_ITEMS,
                           lists + 2 * MASW_NOALLOC_MAX_ITEMS, scan_counters, 1, 0, (int)items, s,
                           nullptr, nullptr);
    if (e != cudaSuccess) return MASW_ECUDA;
    return MASW_OK;
}
