// masw_serve.cu -- continuous-batching request loop for model evaluations.
//
// Repeated evaluation of candidate models is what an inversion or an
// uncertainty sampler does (Section 1; Section 2.1, "exhaustive quantity of
// plausible model parameters"); the paper evaluates one model per call. Here
// requests (one model with its own layer count and wavelengths each) arrive
// at any time and share the GPU:
//  * each admitted request owns a slot: its layer records, wavenumbers, scan
//    state and results stay resident until the request is polled;
//  * admission needs a free slot and room under the byte cap;
//  * every tick runs the counting search over the items (one (request,
//    wavelength) pair each) admitted since the last tick, advances every
//    item still scanning linearly by at most `chunks_per_tick` chunks of
//    Algorithm 1's scan, checks in FP64 what the two located, and compacts
//    the items still running; requests admitted between ticks join the next
//    tick, so their work overlaps with the requests already in flight;
//  * an item's evaluations are exactly those of the batch path (the same
//    search, the same chunks from the same start, sign carried across
//    chunks), so a result does not depend on what else is in flight.
// There are no device-side waits: the host waits for each tick on an event.
//
// Admission builds a request's slot block in one packed pinned upload
// buffer; each tick sends everything admitted since the last tick (blocks,
// their descriptors and the new item ids) with one host-to-device copy, and
// a scatter kernel moves each block into its slot. Slot layout:
//   [meta: 4 x i32 (nrec, nlim, n_lambda, 0)] [records: rmax x 8 f64]
//   [FP32 records: rmax x 8 f32] [k: imax f64]
//   [scan state: imax x (base, carry, phase, located index) i32]
// Each item runs the default scan of the batch path: in the tick after its
// admission, a lane pair runs the counting search (the FP32 negative-
// eigenvalue count split below the pole-free bound) and its FP64 certificate
// (count 0 at V[n-1], odd at V[n]; count_certify_pair), so most requests
// finish in one tick; an uncertified item takes the FP64 search on the
// Wittrick-Williams mode count from V[0] in the same kernel (masw_modes.cuh).
// Items whose change lies above the bound continue with paired FP32 chunks
// from the bound, up to `chunks_per_tick` per tick, and get the batch path's
// three-point FP64 check on the mode count at V[0], V[n-1], V[n]; when it does
// not confirm, the same mode-count search. Items whose FP64 counts fail
// continue with FP64 chunks, one per tick, from V[0].
// Results are written by the kernel into mapped pinned host memory, so
// retiring a request is a host memcpy.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/masw.h"
#include "masw_count.cuh"
#include "masw_device.cuh"
#include "masw_internal.h"
#include "masw_modes.cuh"
#include "masw_screen.cuh"

using namespace masw;

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct SlotView {
    double* region;      // [slots][stride] doubles
    int64_t stride;      // doubles per slot
    int rmax, imax;
    double* ct;          // mapped host [slots * imax]
    int32_t* idx;
    int32_t* status;
    int32_t* remaining;  // [slots] items still running
    int32_t* done;       // [slots] slots finished during the tick
    int32_t* counters;   // [0] survivors, [1] done count, [2] check-list count
    int32_t route;       // test routing (masw_server_set_route), 0 normal
};

__device__ __forceinline__ const int32_t* slot_meta(const SlotView& v, int s) {
    return (const int32_t*)(v.region + (size_t)s * v.stride);
}
__device__ __forceinline__ double* slot_records(const SlotView& v, int s) {
    return v.region + (size_t)s * v.stride + 2;
}
__device__ __forceinline__ float* slot_records32(const SlotView& v, int s) {
    return (float*)(v.region + (size_t)s * v.stride + 2 + (size_t)v.rmax * LAYER_STRIDE);
}
// the certificate's double-float records (LAYER_STRIDE_DF floats a record,
// SLOT_DF doubles)
constexpr int SLOT_DF = LAYER_STRIDE_DF / 2;
__device__ __forceinline__ const float* slot_records_df(const SlotView& v, int s) {
    return (const float*)(v.region + (size_t)s * v.stride + 2 + (size_t)v.rmax * (LAYER_STRIDE + 4));
}
__device__ __forceinline__ double* slot_k(const SlotView& v, int s) {
    return v.region + (size_t)s * v.stride + 2 + (size_t)v.rmax * (LAYER_STRIDE + 4 + SLOT_DF);
}
__device__ __forceinline__ int32_t* slot_state(const SlotView& v, int s) {
    return (int32_t*)(v.region + (size_t)s * v.stride + 2 +
                      (size_t)v.rmax * (LAYER_STRIDE + 4 + SLOT_DF) + v.imax);
}

enum { PH_SCREEN = 0, PH_FP64 = 1 };

// Write an item's result into the mapped host arrays (res < 0: no change
// below the limit) and count it off its request; the request's slot joins
// the done list with its last item.
__device__ __forceinline__ void finish_item(const SlotView& v, int item, int slot, int res,
                                            double c0, double dc) {
    if (res >= 0) {
        v.ct[item] = grid_c(c0, dc, res);
        v.idx[item] = res;
        v.status[item] = MASW_FOUND;
    } else {
        v.ct[item] = __longlong_as_double(0x7ff8000000000000LL);
        v.idx[item] = -1;
        v.status[item] = MASW_NO_ROOT;
    }
    __threadfence_system();
    if (atomicSub(&v.remaining[slot], 1) == 1) v.done[atomicAdd(&v.counters[1], 1)] = slot;
}

// Upload descriptor of one admitted request inside the packed upload buffer.
struct UploadDesc { int32_t slot, offset, bytes, n_lambda; };

// Tick, admission: one block per request copies its block (16-byte words;
// offsets and slot strides are multiples of 256 bytes) from the upload
// buffer into its slot and sets its running-item count.
__global__ void __launch_bounds__(256) serve_scatter_kernel(SlotView v, const unsigned char* __restrict__ up,
                                                            const UploadDesc* __restrict__ desc) {
    const UploadDesc d = desc[blockIdx.x];
    const uint4* src = reinterpret_cast<const uint4*>(up + d.offset);
    uint4* dst = reinterpret_cast<uint4*>(v.region + (size_t)d.slot * v.stride);
    const int words = (d.bytes + 15) / 16;
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) v.remaining[d.slot] = d.n_lambda;
}

// The first change of one item from the FP64 mode-count search from V[0]
// (both lanes of its pair; `topp` is V[nlim-1] when already evaluated, else
// T = -1). Finishes the item and returns true; when the counts fail, queues
// the FP64 scan from V[0] for the next ticks and returns false.
__device__ bool search_or_rescan(SlotView v, int item, int slot, const double* lay, int N,
                                 double k, double c0, double dc, int nlim, TPoint topp, int half,
                                 unsigned pair, int32_t* active_out, const TPoint* p0 = nullptr) {
    TPoint P, dummy;
    if (p0) {
        P = *p0;
    } else {
        eval_pair(slot_records_df(v, slot), lay, N, k, c0, dc, 0, topp.T < 0 ? nlim - 1 : -1, half,
                  pair, &P, &dummy);
        if (topp.T < 0) topp = dummy;
    }
    ModeSearch st = mode_search_init(slot_records_df(v, slot), lay, N, k, c0, dc, nlim - 1, half,
                                     pair, P, topp);
    int d = 0;
    const int n = next_change(st, &d);
    const bool bad = st.bad || v.route >= 3;  // (test routing 3: the FP64 scan for every item)
    if (half) return !bad;
    if (!bad) {
        finish_item(v, item, slot, n, c0, dc);
        return true;
    }
    int32_t* stt = slot_state(v, slot) + 4 * (item - slot * v.imax);
    stt[0] = 0;
    stt[1] = 0;
    stt[2] = PH_FP64;
    active_out[atomicAdd(&v.counters[0], 1)] = item;
    return false;
}

// Tick, part 0 (two lanes per item admitted since the last tick): the
// counting search and its FP64 certificate of the batch path
// (count_certify_pair). A certified item is finished here. When the
// certificate failed, the pair searches the first change on the FP64 mode
// count from V[0] (next_change) and finishes the item too (if those counts
// fail, the FP64 scan from V[0] follows at the next ticks). The fallback
// items continue at the next tick with the linear FP32 screen from the end of
// the pole-free range (carrying the positive sign of count 0) or from V[0].
__global__ void __launch_bounds__(128, 7) serve_count_kernel(SlotView v, const int32_t* __restrict__ items,
                                                             int n_items, int32_t* active_out,
                                                             double c0, double dc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if ((t >> 1) >= n_items) return;  // both lanes of a pair leave together
    const int half = t & 1;
    const unsigned pair = 3u << ((threadIdx.x & 31) & 30);
    const int item = items[t >> 1];
    const int slot = item / v.imax;
    const int j = item - slot * v.imax;
    const int32_t* meta = slot_meta(v, slot);
    const int N = meta[0] - 1;
    const int nlim = meta[1];
    int32_t* stt = slot_state(v, slot) + 4 * j;
    if (nlim < 2) {
        if (!half) finish_item(v, item, slot, -1, c0, dc);
        return;
    }
    const double* lay = slot_records(v, slot);
    const double k = slot_k(v, slot)[j];
    PairCount r =
        count_certify_pair(slot_records32(v, slot), slot_records_df(v, slot), lay, N, k, c0, dc,
                           nlim, half, pair);
    if (v.route >= 1) r = PairCount{-1, -1, 0};  // test routing: the linear screen from V[0]
    if (r.cert >= 1) {
        if (!half) finish_item(v, item, slot, r.cert, c0, dc);
        return;
    }
    if (r.n >= 1) {
        if (search_or_rescan(v, item, slot, lay, N, k, c0, dc, nlim,
                             TPoint{nlim - 1, -1, 0}, half, pair, active_out))
            return;
    } else if (!half) {
        stt[0] = r.start;
        stt[1] = r.start > 0 ? 1 : 0;
        stt[2] = PH_SCREEN;
        active_out[atomicAdd(&v.counters[0], 1)] = item;
    }
}

// Tick, part 1 (one warp per active item). PH_SCREEN: up to `chunks` paired
// FP32 chunks (64 test velocities each); when the screen sees a change (or
// reaches the scan limit) the item goes to the check list with its index.
// PH_FP64: one FP64 chunk (32 test velocities) of the plain scan.
__global__ void __launch_bounds__(256) serve_tick_kernel(SlotView v,
                                                         const int32_t* __restrict__ active_in,
                                                         int n_active, int32_t* active_out,
                                                         int32_t* check_list, int chunks,
                                                         double c0, double dc) {
    extern __shared__ float smemf[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int a = blockIdx.x * (blockDim.x >> 5) + wib;
    if (a >= n_active) return;
    const int item = active_in[a];
    const int slot = item / v.imax;
    const int j = item - slot * v.imax;
    const int32_t* meta = slot_meta(v, slot);
    const int nrec = meta[0];
    const int nlim = meta[1];
    const int N = nrec - 1;
    int32_t* stt = slot_state(v, slot) + 4 * j;
    int base = stt[0], carry = stt[1], phase = stt[2];
    const double k = slot_k(v, slot)[j];
    int res = -1;
    bool finished = false, to_check = false;
    if (phase == PH_SCREEN) {
        float* my = smemf + (size_t)wib * v.rmax * LAYER_STRIDE32;
        const float* src = slot_records32(v, slot);
        for (int t = lane; t < nrec * LAYER_STRIDE32; t += 32) my[t] = src[t];
        __syncwarp();
        const float kf = (float)k, c0f = (float)c0, dcf = (float)dc;
        for (int c = 0; c < chunks && !to_check; ++c) {
            const int n0 = base + 2 * lane, n1 = n0 + 1;
            int s0 = 0, s1 = 0;
            if (n1 < nlim) {
                det_sign_f2(my, N, kf, fmaf((float)n0, dcf, c0f), fmaf((float)n1, dcf, c0f), &s0, &s1);
            } else if (n0 < nlim) {
                s0 = det_sign_f(my, N, kf, fmaf((float)n0, dcf, c0f));
            }
            int prev = __shfl_up_sync(FULL, s1, 1);
            if (lane == 0) prev = carry;
            unsigned m0 = __ballot_sync(FULL, n0 >= 1 && n0 < nlim && s0 != prev);
            unsigned m1 = __ballot_sync(FULL, n1 < nlim && s1 != s0);
            unsigned mm = m0 | m1;
            if (mm) {
                int l = __ffs(mm) - 1;
                res = base + 2 * l + (((m0 >> l) & 1u) ? 0 : 1);
                to_check = true;
            } else {
                carry = __shfl_sync(FULL, s1, 31);
                base += 64;
                if (base >= nlim) { res = -2; to_check = true; }
            }
        }
    } else if (base < nlim) {
        // one FP64 chunk per tick
        const double* lay = slot_records(v, slot);
        int n = base + lane;
        int sg = (n < nlim) ? det_sign(lay, N, k, grid_c(c0, dc, n)) : 0;
        int prev = __shfl_up_sync(FULL, sg, 1);
        if (lane == 0) prev = carry;
        unsigned msk = __ballot_sync(FULL, n >= 1 && n < nlim && sg != prev);
        if (msk) {
            res = base + __ffs(msk) - 1;
            finished = true;
        } else {
            carry = __shfl_sync(FULL, sg, 31);
            base += 32;
            finished = base >= nlim;
        }
    } else {
        finished = true;
    }
    if (lane == 0) {
        if (finished) {
            finish_item(v, item, slot, res, c0, dc);
        } else {
            stt[0] = base;
            stt[1] = carry;
            stt[2] = phase;
            if (to_check) {
                stt[3] = res;  // screen index (-2: none below the limit)
                check_list[atomicAdd(&v.counters[2], 1)] = item;
            } else {
                active_out[atomicAdd(&v.counters[0], 1)] = item;
            }
        }
    }
}

// Tick, part 2 (two lanes per item the linear screen located this tick):
// the three-point check of the batch path on the FP64 mode count
// (mode_count_verified at V[0], V[n-1], V[n], or V[0] and the last point
// when the screen saw no change). An item that fails it takes the FP64
// mode-count search from V[0] in this kernel (search_or_rescan).
__global__ void __launch_bounds__(128) serve_check_kernel(SlotView v,
                                                          const int32_t* __restrict__ check_list,
                                                          const int32_t* __restrict__ n_check,
                                                          int32_t* active_out, double c0, double dc) {
    const int t = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 1);
    const int half = threadIdx.x & 1;
    const unsigned pair = 3u << (threadIdx.x & 30);
    if (t >= *n_check) return;  // both lanes of a pair leave together
    const int item = check_list[t];
    const int slot = item / v.imax;
    const int j = item - slot * v.imax;
    const int32_t* meta = slot_meta(v, slot);
    const int N = meta[0] - 1;
    const int nlim = meta[1];
    if (nlim < 2) {
        if (!half) finish_item(v, item, slot, -1, c0, dc);
        return;
    }
    const double* lay = slot_records(v, slot);
    const double k = slot_k(v, slot)[j];
    const int n = slot_state(v, slot)[4 * j + 3];  // screen index (-2: none below the limit)
    TPoint p0, pa, pb{-1, -1, 0}, unused;
    const float* laydf = slot_records_df(v, slot);
    eval_pair(laydf, lay, N, k, c0, dc, 0, n >= 1 ? n - 1 : nlim - 1, half, pair, &p0, &pa);
    if (n >= 1) eval_pair(laydf, lay, N, k, c0, dc, n, -1, half, pair, &pb, &unused);
    if (v.route < 2 && mode_count_verified(n, p0.T, pa.T, pb.T)) {
        if (!half) finish_item(v, item, slot, n >= 1 ? n : -1, c0, dc);
        return;
    }
    const TPoint topp = n >= 1 ? TPoint{nlim - 1, -1, 0} : pa;
    search_or_rescan(v, item, slot, lay, N, k, c0, dc, nlim, topp, half, pair, active_out, &p0);
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int64_t request_bytes(int32_t n_layers, int32_t n_lambda) {
    // records + per-item k, scan state and results
    return (int64_t)(n_layers + 1) * (LAYER_STRIDE * 8 + LAYER_STRIDE32 * 4 + LAYER_STRIDE_DF * 4) +
           (int64_t)n_lambda * (8 + 16 + 16);
}

int32_t scan_limit_host(const masw_grid& g, double beta_hs) {
    double est = std::floor((beta_hs - g.c0) / g.dc);
    int64_t n = (int64_t)std::max(0.0, std::min(est, (double)g.n_c));
    while (n > 0 && !(std::fma((double)(n - 1), g.dc, g.c0) < beta_hs)) --n;
    while (n < g.n_c && std::fma((double)n, g.dc, g.c0) < beta_hs) ++n;
    return (int32_t)n;
}

}  // namespace

struct masw_server {
    masw_grid grid{};
    masw_server_config cfg{};
    cudaStream_t stream = nullptr;
    SlotView v{};
    // packed upload: [request blocks, 256-byte aligned][descriptors][new item ids]
    unsigned char* h_upload[2] = {nullptr, nullptr};  // pinned, two halves: one staging while
                                                      // the other may still be in a copy
    int up_cur = 0;                                   // half that submit stages into
    unsigned char* d_upload = nullptr;
    size_t upload_cap = 0;   // bytes
    size_t upload_used = 0;  // bytes of request blocks staged since the last tick
    std::vector<UploadDesc> upload_desc;
    double* h_ct = nullptr;      // mapped pinned results
    int32_t* h_idx = nullptr;
    int32_t* h_status = nullptr;
    int32_t* active[2] = {nullptr, nullptr};
    int32_t* check = nullptr;
    int32_t* h_counters = nullptr;
    int32_t* h_done = nullptr;
    cudaEvent_t ev = nullptr;
    int cur = 0;
    int n_active = 0;
    std::vector<int32_t> free_slots;
    std::vector<int64_t> slot_req;  // request id held by a slot (-1 free)
    std::vector<int32_t> slot_nlambda;
    std::vector<int64_t> slot_bytes;
    std::vector<char> slot_done;
    std::vector<int32_t> id_slot;   // request id -> slot (-1 after poll)
    std::vector<int32_t> pending;   // items admitted since the last tick
    std::vector<int32_t> just_done; // slots finished by the last tick
    int64_t bytes_in_flight = 0;
    int32_t pending_active = 0;  // new items of a launched, unfinished tick
    int64_t ticks = 0;
    int64_t completed = 0;
    // opt-in tick profile (masw_server_profile): events between the parts of
    // a tick, accumulated when the tick finishes
    bool prof = false;
    bool prof_pending = false;          // the launched tick recorded its events
    cudaEvent_t pev[6] = {};            // start, scatter, count, tick, check, read-back done
    double prof_acc[MASW_SERVER_PROFILE_VALUES] = {};
};

namespace {

void server_free(masw_server* S) {
    if (!S) return;
    void* dev[] = {S->v.region, S->v.remaining, S->v.counters, S->active[0],
                   S->active[1], S->check, S->d_upload};
    for (void* p : dev)
        if (p) cudaFree(p);
    void* host[] = {S->h_upload[0], S->h_upload[1], S->h_ct, S->h_idx, S->h_status,
                    S->h_counters};
    for (void* p : host)
        if (p) cudaFreeHost(p);
    if (S->ev) cudaEventDestroy(S->ev);
    for (cudaEvent_t e : S->pev)
        if (e) cudaEventDestroy(e);
    delete S;
}

template <typename T>
bool dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}
template <typename T>
bool halloc(T** p, size_t n, unsigned flags = cudaHostAllocDefault) {
    return cudaHostAlloc((void**)p, std::max<size_t>(n, 1) * sizeof(T), flags) == cudaSuccess;
}

// A tick in two halves: tick_launch enqueues the upload of the requests
// admitted since the last tick, the kernels and the copy back of the
// counters and done list, and records the tick's event; tick_finish waits on
// it and takes the finished slots into just_done. Between the two the host
// may admit more requests: they stage into the other half of the upload
// buffer and join the next tick.
int tick_launch_impl(masw_server* S, bool* launched);
int tick_finish_impl(masw_server* S);
int tick_launch(masw_server* S, bool* launched) {
    int rc = tick_launch_impl(S, launched);
    if (rc != MASW_OK) cudaGetLastError();  // leave no pending error behind
    return rc;
}
int tick_finish(masw_server* S) {
    int rc = tick_finish_impl(S);
    if (rc != MASW_OK) cudaGetLastError();
    return rc;
}
int run_tick(masw_server* S) {
    bool launched = false;
    int rc = tick_launch(S, &launched);
    if (rc == MASW_OK && launched) rc = tick_finish(S);
    return rc;
}
// Profile event k of the tick being launched (no-op unless profiling).
bool prof_mark(masw_server* S, int k) {
    return !S->prof || cudaEventRecord(S->pev[k], S->stream) == cudaSuccess;
}
int tick_launch_impl(masw_server* S, bool* launched) {
    *launched = false;
    S->just_done.clear();
    int n_new = (int)S->pending.size();
    if (S->n_active + n_new == 0) return MASW_OK;
    const double t_host = S->prof ? now_s() : 0.0;
    if (!prof_mark(S, 0)) return MASW_ECUDA;
    const int32_t* new_items = nullptr;
    if (n_new) {
        // one transfer: staged blocks, then descriptors, then the new item ids
        unsigned char* up = S->h_upload[S->up_cur];
        const int n_req = (int)S->upload_desc.size();
        const size_t desc_off = S->upload_used;
        const size_t items_off = desc_off + (size_t)n_req * sizeof(UploadDesc);
        const size_t total = items_off + (size_t)n_new * sizeof(int32_t);
        std::memcpy(up + desc_off, S->upload_desc.data(), n_req * sizeof(UploadDesc));
        std::memcpy(up + items_off, S->pending.data(), n_new * sizeof(int32_t));
        if (cudaMemcpyAsync(S->d_upload, up, total, cudaMemcpyHostToDevice, S->stream) !=
            cudaSuccess)
            return MASW_ECUDA;
        serve_scatter_kernel<<<n_req, 256, 0, S->stream>>>(
            S->v, S->d_upload, reinterpret_cast<const UploadDesc*>(S->d_upload + desc_off));
        if (cudaGetLastError() != cudaSuccess) return MASW_ECUDA;
        new_items = reinterpret_cast<const int32_t*>(S->d_upload + items_off);
        S->pending.clear();
        S->upload_desc.clear();
        S->upload_used = 0;
        S->up_cur = 1 - S->up_cur;  // later submits stage into the other half
    }
    if (!prof_mark(S, 1)) return MASW_ECUDA;
    if (cudaMemsetAsync(S->v.counters, 0, 3 * sizeof(int32_t), S->stream) != cudaSuccess)
        return MASW_ECUDA;
    if (n_new) {
        serve_count_kernel<<<(2 * n_new + 127) / 128, 128, 0, S->stream>>>(
            S->v, new_items, n_new, S->active[1 - S->cur], S->grid.c0, S->grid.dc);
        if (cudaGetLastError() != cudaSuccess) return MASW_ECUDA;
    }
    if (!prof_mark(S, 2)) return MASW_ECUDA;
    if (S->n_active) {
        int wpb = S->cfg.warps_per_block;
        int blocks = (S->n_active + wpb - 1) / wpb;
        size_t shm = (size_t)wpb * S->v.rmax * LAYER_STRIDE32 * sizeof(float);
        serve_tick_kernel<<<blocks, 32 * wpb, shm, S->stream>>>(S->v, S->active[S->cur], S->n_active,
                                                                S->active[1 - S->cur], S->check,
                                                                S->cfg.chunks_per_tick, S->grid.c0,
                                                                S->grid.dc);
        if (cudaGetLastError() != cudaSuccess) return MASW_ECUDA;
    }
    if (!prof_mark(S, 3)) return MASW_ECUDA;
    // every item that entered the check list this tick (at most n_active)
    serve_check_kernel<<<(2 * S->n_active + 127) / 128 + 1, 128, 0, S->stream>>>(
        S->v, S->check, S->v.counters + 2, S->active[1 - S->cur], S->grid.c0, S->grid.dc);
    if (cudaGetLastError() != cudaSuccess) return MASW_ECUDA;
    if (!prof_mark(S, 4)) return MASW_ECUDA;
    // counters and the done list (first counters[1] entries) come back together
    if (cudaMemcpyAsync(S->h_counters, S->v.counters, (4 + S->cfg.max_slots) * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
        !prof_mark(S, 5) || cudaEventRecord(S->ev, S->stream) != cudaSuccess)
        return MASW_ECUDA;
    S->pending_active = n_new;  // items of this tick (for the stats until it finishes)
    *launched = true;
    if (S->prof) {
        S->prof_pending = true;
        S->prof_acc[6] += 1e3 * (now_s() - t_host);
    }
    return MASW_OK;
}
int tick_finish_impl(masw_server* S) {
    const double t_host = S->prof ? now_s() : 0.0;
    if (cudaEventSynchronize(S->ev) != cudaSuccess) return MASW_ECUDA;
    if (S->prof_pending) {
        // device time of each part of the tick; the event after the read-back
        // has completed, so every earlier one has too
        for (int k = 0; k < 5; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, S->pev[k], S->pev[k + 1]) != cudaSuccess)
                return MASW_ECUDA;
            S->prof_acc[1 + k] += ms;
        }
        S->prof_acc[0] += 1.0;
        S->prof_acc[7] += 1e3 * (now_s() - t_host);
        S->prof_pending = false;
    }
    int survivors = S->h_counters[0], n_done = S->h_counters[1];
    for (int i = 0; i < n_done; ++i) {
        S->slot_done[S->h_done[i]] = 1;
        S->just_done.push_back(S->h_done[i]);
    }
    S->cur = 1 - S->cur;
    S->n_active = survivors;
    S->pending_active = 0;
    S->ticks++;
    S->completed += n_done;
    return MASW_OK;
}

int slot_of(const masw_server* S, int64_t id) {
    if (id < 0 || id >= (int64_t)S->id_slot.size()) return -1;
    return S->id_slot[id];
}

// Copy a finished slot's results out and free the slot.
void retire_slot(masw_server* S, int slot, double* ct, int32_t* idx, int32_t* status) {
    int n = S->slot_nlambda[slot];
    size_t i0 = (size_t)slot * S->v.imax;
    if (ct) std::memcpy(ct, S->h_ct + i0, n * sizeof(double));
    if (idx) std::memcpy(idx, S->h_idx + i0, n * sizeof(int32_t));
    if (status) std::memcpy(status, S->h_status + i0, n * sizeof(int32_t));
    S->id_slot[S->slot_req[slot]] = -1;
    S->slot_req[slot] = -1;
    S->slot_done[slot] = 0;
    S->bytes_in_flight -= S->slot_bytes[slot];
    S->free_slots.push_back(slot);
}

}  // namespace

extern "C" {

int masw_server_create(const masw_grid* grid, const masw_server_config* cfg, void* cuda_stream,
                       masw_server** out) {
    if (!grid || !cfg || !out) return MASW_EINVAL;
    if (!(std::isfinite(grid->c0) && grid->c0 > 0 && std::isfinite(grid->dc) && grid->dc > 0 &&
          grid->n_c >= 2))
        return MASW_EINVAL;
    if (cfg->max_slots < 1 || cfg->max_layers < 0 || cfg->max_layers > MASW_MAX_LAYERS ||
        cfg->max_lambda < 1 || cfg->mem_cap_bytes <= 0 || cfg->chunks_per_tick < 1 ||
        !(cfg->warps_per_block == 1 || cfg->warps_per_block == 2 || cfg->warps_per_block == 4 ||
          cfg->warps_per_block == 8))
        return MASW_EINVAL;
    int64_t cap_items = (int64_t)cfg->max_slots * cfg->max_lambda;
    if (cap_items > INT32_MAX / 2) return MASW_EINVAL;
    size_t shm = (size_t)cfg->warps_per_block * (cfg->max_layers + 1) * LAYER_STRIDE32 * 4;
    if (shm > 48 * 1024) return MASW_EINVAL;
    masw_server* S = new (std::nothrow) masw_server();
    if (!S) return MASW_ENOMEM;
    S->grid = *grid;
    S->cfg = *cfg;
    S->stream = (cudaStream_t)cuda_stream;
    S->v.rmax = cfg->max_layers + 1;
    S->v.imax = cfg->max_lambda;
    S->v.stride = 2 + (int64_t)S->v.rmax * (LAYER_STRIDE + 4 + SLOT_DF) + 3 * (int64_t)S->v.imax;
    S->v.stride = (S->v.stride + 31) / 32 * 32;  // 256-byte aligned slots
    size_t slots = cfg->max_slots, items = (size_t)cap_items;
    // every slot's block at once, plus descriptors and item ids
    S->upload_cap = slots * (size_t)S->v.stride * sizeof(double) + slots * sizeof(UploadDesc) +
                    items * sizeof(int32_t) + 256;
    if (S->upload_cap > (size_t)INT32_MAX) {  // upload offsets are 32-bit
        server_free(S);
        return MASW_EINVAL;
    }
    // counters (3, padded to 4) and the done list share one buffer: one copy back per tick
    bool ok = dalloc(&S->v.region, slots * S->v.stride) && dalloc(&S->v.remaining, slots) &&
              dalloc(&S->v.counters, 4 + slots) &&
              dalloc(&S->active[0], items) && dalloc(&S->active[1], items) &&
              dalloc(&S->check, items) && dalloc(&S->d_upload, S->upload_cap) &&
              halloc(&S->h_upload[0], S->upload_cap) && halloc(&S->h_upload[1], S->upload_cap) &&
              halloc(&S->h_ct, items, cudaHostAllocMapped) &&
              halloc(&S->h_idx, items, cudaHostAllocMapped) &&
              halloc(&S->h_status, items, cudaHostAllocMapped) &&
              halloc(&S->h_counters, 4 + slots) &&
              cudaEventCreateWithFlags(&S->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&S->v.ct, S->h_ct, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&S->v.idx, S->h_idx, 0) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&S->v.status, S->h_status, 0) == cudaSuccess;
    if (ok) {
        S->v.done = S->v.counters + 4;
        S->h_done = S->h_counters + 4;
    }
    if (!ok) {
        cudaGetLastError();
        server_free(S);
        return MASW_ENOMEM;
    }
    S->free_slots.resize(slots);
    for (size_t s = 0; s < slots; ++s) S->free_slots[s] = (int32_t)(slots - 1 - s);
    S->slot_req.assign(slots, -1);
    S->slot_nlambda.assign(slots, 0);
    S->slot_bytes.assign(slots, 0);
    S->slot_done.assign(slots, 0);
    *out = S;
    return MASW_OK;
}

int masw_server_destroy(masw_server* S) {
    if (!S) return MASW_EINVAL;
    cudaStreamSynchronize(S->stream);
    server_free(S);
    return MASW_OK;
}

static int server_submit(masw_server* S, int32_t n_layers, const double* h, const double* alpha,
                         const double* beta, const double* rho, int32_t n_lambda,
                         const double* lambda, int64_t* request_id);

int masw_server_submit(masw_server* S, int32_t n_layers, const double* h, const double* alpha,
                       const double* beta, const double* rho, int32_t n_lambda,
                       const double* lambda, int64_t* request_id) {
    if (!S || !S->prof) return server_submit(S, n_layers, h, alpha, beta, rho, n_lambda, lambda,
                                             request_id);
    const double t = now_s();
    const int rc = server_submit(S, n_layers, h, alpha, beta, rho, n_lambda, lambda, request_id);
    S->prof_acc[8] += 1e3 * (now_s() - t);
    return rc;
}

int masw_server_profile(masw_server* S, int32_t enable, double* out) {
    if (!S || (enable != 0 && enable != 1)) return MASW_EINVAL;
    if (enable && !S->prof) {
        if (cudaStreamSynchronize(S->stream) != cudaSuccess) return MASW_ECUDA;
        for (cudaEvent_t& e : S->pev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) return MASW_ECUDA;
        for (double& v : S->prof_acc) v = 0.0;
        S->prof_pending = false;
    }
    S->prof = enable == 1;
    if (out)
        for (int k = 0; k < MASW_SERVER_PROFILE_VALUES; ++k) out[k] = S->prof_acc[k];
    return MASW_OK;
}

static int server_submit(masw_server* S, int32_t n_layers, const double* h, const double* alpha,
                         const double* beta, const double* rho, int32_t n_lambda,
                         const double* lambda, int64_t* request_id) {
    if (!S || !alpha || !beta || !rho || !lambda || !request_id || (n_layers > 0 && !h))
        return MASW_EINVAL;
    if (n_layers < 0 || n_layers > S->cfg.max_layers || n_lambda < 1 || n_lambda > S->v.imax)
        return MASW_EINVAL;
    for (int i = 0; i < n_layers; ++i)
        if (!(std::isfinite(h[i]) && h[i] > 0)) return MASW_EINVAL;
    for (int i = 0; i <= n_layers; ++i) {
        double a = alpha[i], b = beta[i], r = rho[i];
        if (!(std::isfinite(a) && a > 0 && std::isfinite(b) && b > 0 && std::isfinite(r) && r > 0 &&
              3.0 * a * a > 4.0 * b * b))
            return MASW_EINVAL;
    }
    for (int j = 0; j < n_lambda; ++j)
        if (!(std::isfinite(lambda[j]) && lambda[j] > 0)) return MASW_EINVAL;
    int64_t need = request_bytes(n_layers, n_lambda);
    if (S->free_slots.empty() || S->bytes_in_flight + need > S->cfg.mem_cap_bytes) return MASW_EADMIT;
    int slot = S->free_slots.back();
    // build meta, records (as masw_model_batch_create builds them), k and a
    // zero scan state in the packed upload buffer; the next tick sends it
    double* reg = reinterpret_cast<double*>(S->h_upload[S->up_cur] + S->upload_used);
    int32_t* meta = (int32_t*)reg;
    meta[0] = n_layers + 1;
    meta[1] = scan_limit_host(S->grid, beta[n_layers]);
    meta[2] = n_lambda;
    meta[3] = 0;
    double* rec = reg + 2;
    for (int i = 0; i <= n_layers; ++i) {
        double* L = rec + (size_t)i * LAYER_STRIDE;
        double a = alpha[i], b = beta[i], r = rho[i];
        L[L_H] = (i < n_layers) ? h[i] : 0.0;
        L[L_MU] = r * b * b;
        L[L_RHO] = r;
        L[L_IA2] = 1.0 / (a * a);
        L[L_IB2] = 1.0 / (b * b);
        L[L_BETA] = b;
        L[L_RATIO] = a / b;
        L[L_IRHO] = 1.0 / r;
    }
    // FP32 records of the screen (stiffnesses over the half-space shear modulus)
    float* rec32 = (float*)(rec + (size_t)S->v.rmax * LAYER_STRIDE);
    double mref = rec[(size_t)n_layers * LAYER_STRIDE + L_MU];
    for (int i = 0; i <= n_layers; ++i) {
        const double* L = rec + (size_t)i * LAYER_STRIDE;
        float* F = rec32 + (size_t)i * LAYER_STRIDE32;
        F[F_H] = (float)L[L_H];
        F[F_MU] = (float)(L[L_MU] / mref);
        F[F_RHO] = (float)(L[L_RHO] / mref);
        F[F_IA2] = (float)L[L_IA2];
        F[F_IB2] = (float)L[L_IB2];
        F[F_DIB] = (float)(L[L_IB2] - L[L_IA2]);
        F[6] = F[7] = 0.0f;
    }
    // the certificate's double-float records
    float* recdf = (float*)(rec + (size_t)S->v.rmax * (LAYER_STRIDE + 4));
    for (int i = 0; i <= n_layers; ++i)
        df_record(rec + (size_t)i * LAYER_STRIDE, recdf + (size_t)i * LAYER_STRIDE_DF);
    double* kk = rec + (size_t)S->v.rmax * (LAYER_STRIDE + 4 + SLOT_DF);
    for (int j = 0; j < n_lambda; ++j) kk[j] = 2.0 * M_PI / lambda[j];
    int32_t* stt = (int32_t*)(kk + S->v.imax);
    std::memset(stt, 0, (size_t)n_lambda * 4 * sizeof(int32_t));
    const size_t bytes = (size_t)((char*)(stt + 4 * n_lambda) - (char*)reg);
    S->upload_desc.push_back({slot, (int32_t)S->upload_used, (int32_t)bytes, n_lambda});
    S->upload_used += (bytes + 255) / 256 * 256;
    S->free_slots.pop_back();
    int64_t id = (int64_t)S->id_slot.size();
    S->id_slot.push_back(slot);
    int64_t i0 = (int64_t)slot * S->v.imax;
    for (int j = 0; j < n_lambda; ++j) S->pending.push_back((int32_t)(i0 + j));
    S->slot_req[slot] = id;
    S->slot_nlambda[slot] = n_lambda;
    S->slot_bytes[slot] = need;
    S->slot_done[slot] = 0;
    S->bytes_in_flight += need;
    *request_id = id;
    return MASW_OK;
}

int masw_server_tick(masw_server* S, int32_t* n_completed) {
    if (!S) return MASW_EINVAL;
    int rc = run_tick(S);
    if (rc) return rc;
    if (n_completed) *n_completed = (int32_t)S->just_done.size();
    return MASW_OK;
}

int masw_server_poll(masw_server* S, int64_t request_id, double* ct, int32_t* ct_idx,
                     int32_t* status) {
    if (!S) return MASW_EINVAL;
    int slot = slot_of(S, request_id);
    if (slot < 0) return MASW_EINVAL;
    if (!S->slot_done[slot]) return MASW_EAGAIN;
    retire_slot(S, slot, ct, ct_idx, status);
    return MASW_OK;
}

int masw_server_set_route(masw_server* S, int32_t route) {
    if (!S || route < 0 || route > 3) return MASW_EINVAL;
    S->v.route = route;
    return MASW_OK;
}

int masw_server_get_stats(const masw_server* S, masw_server_stats* st) {
    if (!S || !st) return MASW_EINVAL;
    st->in_flight = (int32_t)(S->cfg.max_slots - (int32_t)S->free_slots.size());
    st->active_items = S->n_active + S->pending_active + (int32_t)S->pending.size();
    st->bytes_in_flight = S->bytes_in_flight;
    st->ticks = S->ticks;
    st->completed = S->completed;
    return MASW_OK;
}

int masw_server_run_trace(masw_server* S, int32_t n_requests, const int32_t* n_layers,
                          const double* h, const double* alpha, const double* beta,
                          const double* rho, const int32_t* n_lambda, const double* lambda,
                          const double* arrival_s, double timeout_s, double* latency_s,
                          double* ct, int32_t* ct_idx, int32_t* status, int64_t* stats) {
    if (!S || n_requests < 1 || !n_layers || !alpha || !beta || !rho || !n_lambda || !lambda ||
        !arrival_s || !latency_s)
        return MASW_EINVAL;
    if (S->free_slots.size() != (size_t)S->cfg.max_slots) return MASW_EINVAL;  // must start idle
    std::vector<int64_t> hoff(n_requests + 1, 0), loff(n_requests + 1, 0), woff(n_requests + 1, 0);
    for (int i = 0; i < n_requests; ++i) {
        if (n_layers[i] < 0 || n_lambda[i] < 1) return MASW_EINVAL;
        hoff[i + 1] = hoff[i] + n_layers[i];
        loff[i + 1] = loff[i] + n_layers[i] + 1;
        woff[i + 1] = woff[i] + n_lambda[i];
        if (i && arrival_s[i] < arrival_s[i - 1]) return MASW_EINVAL;
    }
    std::vector<int32_t> slot_q(S->cfg.max_slots, -1);
    int next = 0, done = 0;
    int64_t refused = 0, max_in_flight = 0;
    bool blocked = false;  // the next arrival was refused: wait for a tick to free room
    const double t0 = now_s();
    // admit every request that has arrived, while slots and bytes allow
    auto admit = [&]() -> int {
        double t = now_s() - t0;
        while (next < n_requests && arrival_s[next] <= t && !blocked) {
            int64_t id;
            int rc = masw_server_submit(S, n_layers[next], h + hoff[next], alpha + loff[next],
                                        beta + loff[next], rho + loff[next], n_lambda[next],
                                        lambda + woff[next], &id);
            if (rc == MASW_EADMIT) {
                ++refused;
                blocked = true;
                break;
            }
            if (rc) return rc;
            slot_q[S->id_slot[id]] = next;
            ++next;
        }
        max_in_flight =
            std::max<int64_t>(max_in_flight, S->cfg.max_slots - (int64_t)S->free_slots.size());
        return MASW_OK;
    };
    while (done < n_requests) {
        if (now_s() - t0 > timeout_s) return MASW_ETIMEOUT;
        int rc = admit();
        if (rc) return rc;
        bool launched = false;
        if ((rc = tick_launch(S, &launched))) return rc;
        if (launched) {
            // the GPU runs the tick; keep admitting into the other upload half
            while (cudaEventQuery(S->ev) == cudaErrorNotReady) {
                if ((rc = admit())) return rc;
                if (now_s() - t0 > timeout_s) return MASW_ETIMEOUT;
            }
            if ((rc = tick_finish(S))) return rc;
            blocked = false;
            double tc = now_s() - t0;
            for (int slot : S->just_done) {
                int q = slot_q[slot];
                slot_q[slot] = -1;
                retire_slot(S, slot, ct ? ct + woff[q] : nullptr, ct_idx ? ct_idx + woff[q] : nullptr,
                            status ? status + woff[q] : nullptr);
                latency_s[q] = tc - arrival_s[q];
                ++done;
            }
        } else if (next < n_requests) {
            blocked = false;
            double wait = arrival_s[next] - (now_s() - t0);
            if (wait > 0)
                std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 1e-3)));
        }
    }
    if (stats) {
        stats[0] = S->ticks;
        stats[1] = refused;
        stats[2] = max_in_flight;
    }
    return MASW_OK;
}

}  // extern "C"
