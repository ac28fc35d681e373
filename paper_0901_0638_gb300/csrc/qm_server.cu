// qm_server.cu -- continuous-batching server for Monte Carlo sample requests.
//
// Native host engine:
//   * a device arena (one cudaMalloc of the memory budget at create) with a
//     first-fit host-side allocator: a request is admitted only when its
//     output fits, and its bytes stay allocated until the caller releases
//     them (outputs stay on the device);
//   * a worker thread that, in a loop, (1) retires finished batches (event
//     queries), (2) admits pending requests in FIFO order while memory, batch
//     and stream slots allow, (3) packs the admitted requests into a request
//     table and launches one kernel for all of them on a free stream.  New
//     arrivals are admitted while earlier batches run, and batches on
//     different streams overlap on the device;
//   * "plain" mode (one request per launch, one stream) is the baseline.
// Every wait is bounded; an expired wait returns QM_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qm.h"
#include "qm_device.cuh"
#include "qm_fx.cuh"
#include "qm_host.h"

namespace qm {

struct ReqDev {
    void* out;
    unsigned long long n;
    unsigned long long key;
    unsigned long long tile0;
    int kind;
    int pad;
    TSel t;
};

constexpr int kServeBlock = 256;
constexpr int kServePhilox = 4;                             // Philox blocks per thread
constexpr int kServeTile = kServeBlock * kServePhilox;     // Philox blocks per tile

__device__ __forceinline__ void serve_f32(const ReqDev& r, unsigned long long pb)
{
    const uint4 w = philox_block(r.key, pb);
    const unsigned long long i0 = pb * 4;
    float* o = static_cast<float*>(r.out);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    if (i0 + 4 <= r.n && ((uintptr_t)(o + i0) % 16 == 0)) {
        __stcs(reinterpret_cast<float4*>(o + i0),
               make_float4(probit_grid24_tbl(ws[0] >> 8), probit_grid24_tbl(ws[1] >> 8),
                           probit_grid24_tbl(ws[2] >> 8), probit_grid24_tbl(ws[3] >> 8)));
    } else {
        for (int j = 0; j < 4; ++j)
            if (i0 + j < r.n) o[i0 + j] = probit_grid24_tbl(ws[j] >> 8);
    }
}

__device__ __forceinline__ double serve_f64_one(const fxt::FxTable* fxT, int kind, const TSel& t, uint32_t hi,
                                                uint32_t lo)
{
    const uint64_t k = ((uint64_t)(hi >> 11) << 32) | lo;
    bool upper;
    const double m = probit_grid53_fx<FX_FP64_LEAN>(fxT, k, upper);      // |Phi^{-1}((k + 1/2) 2^-53)|
    if (kind == 3) {
        // Exp(1) sample x = -log(u), u = (k + 1/2) 2^-53, recycled to the
        // normal by Q(x) = Phi^{-1}(1 - e^{-x}) = Phi^{-1}(1 - u) (Sec. 6): the
        // exponential coordinate of u is evaluated by the table from u's bits,
        // so x is never rounded (z > 0 exactly when u < 1/2).
        return __longlong_as_double(__double_as_longlong(m) ^ (long long)((unsigned long long)upper << 63));
    }
    // the sign on the bits (a select between m and -m costs FP64 instructions)
    const double z = __longlong_as_double(__double_as_longlong(m) ^ (long long)((unsigned long long)!upper << 63));
    if (kind == 2) return recycle_t_call(t, z);
    return z;
}

__global__ void __launch_bounds__(kServeBlock)
k_serve(const ReqDev* __restrict__ reqs, int nreq, unsigned long long ntiles, const fxt::FxTable* fxT)
{
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int lo = 0, hi = nreq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (reqs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
        }
        const ReqDev r = reqs[lo];
        const unsigned long long per = (r.kind == 0) ? 4 : 2;      // samples per Philox block
        const unsigned long long nblk = (r.n + per - 1) / per;
        const unsigned long long b0 = (tile - r.tile0) * kServeTile;
#pragma unroll
        for (int k = 0; k < kServePhilox; ++k) {
            const unsigned long long pb = b0 + (unsigned long long)k * kServeBlock + threadIdx.x;
            if (pb >= nblk) continue;
            if (r.kind == 0) {
                serve_f32(r, pb);
            } else {
                const uint4 w = philox_block(r.key, pb);
                double* o = static_cast<double*>(r.out);
                const double z0 = serve_f64_one(fxT, r.kind, r.t, w.x, w.y);
                const double z1 = serve_f64_one(fxT, r.kind, r.t, w.z, w.w);
                const unsigned long long i0 = pb * 2;
                if (i0 + 2 <= r.n && ((uintptr_t)(o + i0) % 16 == 0)) {
                    __stcs(reinterpret_cast<double2*>(o + i0), make_double2(z0, z1));
                } else {
                    if (i0 < r.n) o[i0] = z0;
                    if (i0 + 1 < r.n) o[i0 + 1] = z1;
                }
            }
        }
    }
}

static unsigned long long req_tiles(const ReqDev& r)
{
    const unsigned long long per = (r.kind == 0) ? 4 : 2;
    const unsigned long long nblk = (r.n + per - 1) / per;
    return (nblk + kServeTile - 1) / kServeTile;
}

// ----------------------------------------------------------------------------
// Device arena: first-fit over free extents, 256-byte granularity.
// ----------------------------------------------------------------------------
class Arena {
public:
    bool init(size_t bytes)
    {
        cap_ = (bytes + 255) & ~(size_t)255;
        if (cudaMalloc(&base_, cap_) != cudaSuccess) return false;
        free_[0] = cap_;
        return true;
    }
    void destroy()
    {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    void* alloc(size_t bytes)
    {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                sizes_[off] = bytes;
                return (char*)base_ + off;
            }
        }
        return nullptr;
    }
    void release(void* p)
    {
        const size_t off = (char*)p - (char*)base_;
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t len = s->second;
        sizes_.erase(s);
        used_ -= len;
        size_t start = off;
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        next = free_.lower_bound(start + len);
        if (next != free_.end() && next->first == start + len) {
            len += next->second;
            free_.erase(next);
        }
        free_[start] = len;
    }
    size_t used() const { return used_; }
    size_t capacity() const { return cap_; }

private:
    void* base_ = nullptr;
    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
    std::map<size_t, size_t> sizes_;
};

}  // namespace qm

using namespace qm;

struct qm_server {
    qm_server_config cfg{};
    Arena arena;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<qm_request> pending;
    std::deque<qm_completion> done;
    std::unordered_map<uint64_t, void*> held;      // id -> output (until released)
    std::vector<uint64_t> to_release;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    // per stream slot
    struct Slot {
        cudaStream_t stream = nullptr;
        cudaEvent_t ev = nullptr;
        ReqDev* host = nullptr;      // pinned
        ReqDev* dev = nullptr;
        std::vector<qm_completion> members;
        bool busy = false;
    };
    std::vector<Slot> slots;
    size_t launches = 0;
    qm_status error = QM_OK;
    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace qm {

static size_t req_bytes(const qm_request& r)
{
    return r.n * (r.kind == QM_REQ_NORMAL_F32 ? 4 : 8);
}

static void worker_loop(qm_server* s)
{
    cudaSetDevice(s->cfg.device);
    const int sms = sm_count() > 0 ? sm_count() : 1;
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_serve, kServeBlock, 0);
    if (bps < 1) bps = 1;
    qm_status fst;
    const fxt::FxTable* fxT = (const fxt::FxTable*)fx_table_device(&fst);   // looked up at create
    std::vector<ReqDev> table;
    while (true) {
        bool idle = true;
        // (1) retire finished batches
        for (auto& sl : s->slots) {
            if (sl.busy && cudaEventQuery(sl.ev) == cudaSuccess) {
                const double t = s->now();
                std::lock_guard<std::mutex> lk(s->mu);
                for (auto& c : sl.members) {
                    c.t_done = t;
                    if (s->cfg.release_on_done) {
                        s->arena.release(c.out);
                        c.out = nullptr;
                    } else {
                        s->held[c.id] = c.out;
                    }
                    s->done.push_back(c);
                }
                sl.members.clear();
                sl.busy = false;
                idle = false;
                s->cv.notify_all();
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (uint64_t id : s->to_release) {
                auto it = s->held.find(id);
                if (it != s->held.end()) {
                    s->arena.release(it->second);
                    s->held.erase(it);
                }
            }
            s->to_release.clear();
        }
        // (2) admit into a free slot and (3) launch
        for (auto& sl : s->slots) {
            if (sl.busy) continue;
            std::vector<qm_completion> batch;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                while (!s->pending.empty() && (int)batch.size() < s->cfg.max_batch) {
                    const qm_request& r = s->pending.front();
                    void* p = r.n ? s->arena.alloc(req_bytes(r)) : nullptr;
                    if (r.n && !p) break;                    // FIFO: wait for memory
                    qm_completion c{};
                    c.id = r.id;
                    c.status = QM_OK;
                    c.out = p;
                    c.n = r.n;
                    c.is_f64 = r.kind != QM_REQ_NORMAL_F32;
                    c.t_arrival = r.t_arrival;
                    c.t_admit = s->now();
                    c.kind = r.kind;
                    c.nu = r.nu;
                    c.key = r.key;
                    batch.push_back(c);
                    s->pending.pop_front();
                }
            }
            if (batch.empty()) break;
            idle = false;
            table.clear();
            unsigned long long t0 = 0;
            for (auto& c : batch) {
                ReqDev d{};
                d.out = c.out;
                d.n = c.n;
                d.key = c.key;
                d.kind = c.kind;
                d.t.k = 0;
                if (c.kind == QM_REQ_STUDENT_T) {
                    const void* tseg = nullptr;
                    const double* ttail = nullptr;
                    t_select(c.nu, &d.t.k, &tseg, &ttail);   // validated (and built) at submit
                    d.t.seg = (const ttbl::TRows*)tseg;
                    d.t.tail = ttail;
                }
                d.tile0 = t0;
                t0 += req_tiles(d);
                table.push_back(d);
            }
            std::memcpy(sl.host, table.data(), sizeof(ReqDev) * table.size());
            cudaMemcpyAsync(sl.dev, sl.host, sizeof(ReqDev) * table.size(), cudaMemcpyHostToDevice, sl.stream);
            const double tl = s->now();
            for (auto& c : batch) c.t_launch = tl;
            if (t0 > 0) {
                const int grid = (int)std::min<unsigned long long>(t0, (unsigned long long)sms * bps);
                k_serve<<<grid, kServeBlock, 0, sl.stream>>>(sl.dev, (int)table.size(), t0, fxT);
            }
            cudaEventRecord(sl.ev, sl.stream);
            if (cudaGetLastError() != cudaSuccess) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->error = QM_ERR_CUDA;
            }
            sl.members = std::move(batch);
            sl.busy = true;
            ++s->launches;
        }
        if (s->stop.load()) {
            bool any = false;
            for (auto& sl : s->slots) any |= sl.busy;
            std::lock_guard<std::mutex> lk(s->mu);
            if (!any && s->pending.empty()) break;
        }
        if (idle) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace qm

extern "C" qm_status qm_server_create(const qm_server_config* cfg, qm_server** out)
{
    if (!cfg || !out) return fail(QM_ERR_INVALID, "qm_server_create: null argument");
    *out = nullptr;
    if (cfg->mem_budget == 0 || cfg->max_batch < 1 || cfg->streams < 1 || cfg->streams > 8)
        return fail(QM_ERR_INVALID, "qm_server_create: budget > 0, max_batch >= 1, 1 <= streams <= 8");
    qm_server* s = new (std::nothrow) qm_server;
    if (!s) return fail(QM_ERR_NOMEM, "qm_server_create: host allocation failed");
    s->cfg = *cfg;
    if (cudaSetDevice(cfg->device) != cudaSuccess) {
        delete s;
        return fail(QM_ERR_CUDA, "qm_server_create: cudaSetDevice(%d) failed", cfg->device);
    }
    {
        qm_status fst;
        if (!fx_table_device(&fst)) {                 // the worker's kernels read this table
            delete s;
            return fst;
        }
        // the offline Student-t tables (converted to their device form at
        // first use) are built here, not at the first Student-t request
        int tk = 0;
        const void* tseg = nullptr;
        const double* ttail = nullptr;
        const qm_status tst = t_select(ttbl::T_NU[0], &tk, &tseg, &ttail);
        if (tst != QM_OK) {
            delete s;
            return tst;
        }
    }
    if (!s->arena.init(cfg->mem_budget)) {
        delete s;
        return fail(QM_ERR_NOMEM, "qm_server_create: device arena of %zu bytes failed", cfg->mem_budget);
    }
    s->slots.resize(cfg->streams);
    for (auto& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.host, sizeof(ReqDev) * cfg->max_batch) != cudaSuccess ||
            cudaMalloc(&sl.dev, sizeof(ReqDev) * cfg->max_batch) != cudaSuccess) {
            qm_server_destroy(s);
            return fail(QM_ERR_NOMEM, "qm_server_create: stream slot setup failed");
        }
    }
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return QM_OK;
}

extern "C" double qm_server_now(const qm_server* s) { return s ? s->now() : 0.0; }

extern "C" qm_status qm_server_submit(qm_server* s, const qm_request* r)
{
    if (!s || !r) return fail(QM_ERR_INVALID, "qm_server_submit: null argument");
    if (r->kind < QM_REQ_NORMAL_F32 || r->kind > QM_REQ_EXP_NORMAL)
        return fail(QM_ERR_INVALID, "qm_server_submit: bad kind %d", r->kind);
    if (r->kind == QM_REQ_STUDENT_T) {
        int k;
        const void* tseg;
        const double* ttail;
        const qm_status st = t_select(r->nu, &k, &tseg, &ttail);   // builds untabulated tables here
        if (st != QM_OK) return st;
    }
    const size_t bytes = r->n * (r->kind == QM_REQ_NORMAL_F32 ? 4 : 8);
    if (bytes > s->arena.capacity())
        return fail(QM_ERR_NOMEM, "qm_server_submit: request of %zu bytes exceeds the budget", bytes);
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.push_back(*r);
    s->cv.notify_all();
    return QM_OK;
}

extern "C" qm_status qm_server_poll(qm_server* s, qm_completion* out, int max, int* got)
{
    if (!s || !got || (max > 0 && !out)) return fail(QM_ERR_INVALID, "qm_server_poll: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *got = k;
    return s->error;
}

extern "C" qm_status qm_server_release(qm_server* s, uint64_t id)
{
    if (!s) return fail(QM_ERR_INVALID, "qm_server_release: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    s->to_release.push_back(id);
    s->cv.notify_all();
    return QM_OK;
}

extern "C" qm_status qm_server_stats(const qm_server* s, qm_server_stats_t* st)
{
    if (!s || !st) return fail(QM_ERR_INVALID, "qm_server_stats: null argument");
    st->launches = s->launches;
    st->arena_used = s->arena.used();
    st->arena_capacity = s->arena.capacity();
    return QM_OK;
}

// Replays `trace` in real time (each request submitted at its t_arrival,
// seconds from the call), waits for all completions (bounded by
// timeout_s) and returns them in `out` (nreq entries, completion order).
extern "C" qm_status qm_server_replay(qm_server* s, const qm_request* trace, int nreq, double timeout_s,
                                     qm_completion* out)
{
    if (!s || (nreq > 0 && (!trace || !out))) return fail(QM_ERR_INVALID, "qm_server_replay: null argument");
    const double start = s->now();
    int next = 0, collected = 0;
    while (collected < nreq) {
        const double t = s->now() - start;
        while (next < nreq && trace[next].t_arrival <= t) {
            qm_request r = trace[next];
            r.t_arrival = start + trace[next].t_arrival;
            const qm_status st = qm_server_submit(s, &r);
            if (st != QM_OK) return st;
            ++next;
        }
        int got = 0;
        const qm_status pst = qm_server_poll(s, out + collected, nreq - collected, &got);
        if (pst != QM_OK) return fail(pst, "qm_server_replay: device error in a batch");
        collected += got;
        if (t > timeout_s) return fail(QM_ERR_TIMEOUT, "qm_server_replay: %d of %d done after %.1f s",
                                       collected, nreq, timeout_s);
        if (got == 0) {
            const double wait = next < nreq ? trace[next].t_arrival - t : 1e-4;
            if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds(100));
            else std::this_thread::yield();
        }
    }
    return QM_OK;
}

extern "C" qm_status qm_server_destroy(qm_server* s)
{
    if (!s) return QM_OK;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    s->arena.destroy();
    delete s;
    return QM_OK;
}
