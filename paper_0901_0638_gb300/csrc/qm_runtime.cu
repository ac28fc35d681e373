// qm_runtime.cu -- ragged batches of recycling jobs: one persistent launch
// over a device-resident segment table, replayed as a CUDA graph, with an
// autotuner over (block size, elements per thread, Horner vs Estrin).
//
// Layout: every segment is cut into tiles of block x ept elements; a tile
// never spans two segments, so the target (and nu) is uniform per block.
// tile0[s] is the prefix sum of the segments' tile counts; a block finds the
// segment of its first tile by binary search over that array and, as its
// tiles increase, steps forward from there.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "qm.h"
#include "qm_device.cuh"
#include "qm_fx.cuh"
#include "qm_exp_map.cuh"
#include "qm_host.h"

namespace qm {

enum { KIND_T = 0, KIND_EXP = 1, KIND_UNIFORM = 2 };

struct DevSeg {
    const double* in;
    double* out;
    unsigned long long n;
    unsigned long long tile0;
    int kind;
    int pad;
    TSel t;
};

template <int EPT, bool ESTRIN>
__global__ void __launch_bounds__(512)
k_batch(const DevSeg* __restrict__ segs, int nseg, unsigned long long ntiles, const fxt::FxTable* fxT)
{
    // the block's tiles increase, so after a binary search for its first
    // tile the segment index only moves forward (segments of zero tiles,
    // equal tile0, are stepped over)
    int lo = 0;
    if (blockIdx.x < ntiles) {
        int hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (segs[mid].tile0 <= blockIdx.x) lo = mid; else hi = mid - 1;
        }
    }
    for (unsigned long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        while (lo + 1 < nseg && segs[lo + 1].tile0 <= tile) ++lo;
        const DevSeg sg = segs[lo];
        const size_t base = (size_t)(tile - sg.tile0) * blockDim.x * EPT;
        // values move as bits: a select or a join of doubles costs FP64
        // instructions, and the maps are bound by that pipe
        unsigned long long xb[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const size_t i = base + (size_t)k * blockDim.x + threadIdx.x;
            xb[k] = (i < sg.n) ? (unsigned long long)__ldcs(reinterpret_cast<const long long*>(sg.in) + i) : 0ull;
        }
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const size_t i = base + (size_t)k * blockDim.x + threadIdx.x;
            const double x = __longlong_as_double((long long)xb[k]);
            long long y;
            if (sg.kind == KIND_T) y = __double_as_longlong(recycle_t_sel<ESTRIN>(sg.t, x));
            else if (sg.kind == KIND_EXP) y = __double_as_longlong(exp_to_normal_fx(x));
            else y = __double_as_longlong(probit_fx<FX_FP64_LEAN>(fxT, x));
            if (i < sg.n) __stcs(reinterpret_cast<long long*>(sg.out) + i, y);
        }
    }
}

// One plain launch per segment (the comparison baseline for the batch).
__global__ void __launch_bounds__(256)
k_single(const double* __restrict__ in, double* out, size_t n, int kind, TSel t, const fxt::FxTable* fxT)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double x = __ldcs(in + i);
        long long y;                                   // as bits (see k_batch)
        if (kind == KIND_T) y = __double_as_longlong(recycle_t_sel<false>(t, x));
        else if (kind == KIND_EXP) y = __double_as_longlong(exp_to_normal_fx(x));
        else y = __double_as_longlong(probit_fx<FX_FP64_LEAN>(fxT, x));
        __stcs(reinterpret_cast<long long*>(out) + i, y);
    }
}

using BatchKernel = void (*)(const DevSeg*, int, unsigned long long, const fxt::FxTable*);

static BatchKernel pick_kernel(int ept, int estrin)
{
    if (estrin) {
        if (ept == 1) return k_batch<1, true>;
        if (ept == 2) return k_batch<2, true>;
        return k_batch<4, true>;
    }
    if (ept == 1) return k_batch<1, false>;
    if (ept == 2) return k_batch<2, false>;
    return k_batch<4, false>;
}

static bool valid_tuning(const qm_tuning& t)
{
    return (t.block == 128 || t.block == 256 || t.block == 512) &&
           (t.ept == 1 || t.ept == 2 || t.ept == 4) && (t.estrin == 0 || t.estrin == 1);
}

}  // namespace qm

using namespace qm;

struct qm_batch {
    std::vector<DevSeg> host;      // kind/tk/in/out/n as created
    DevSeg* dev = nullptr;
    int nseg = 0;
    unsigned long long ntiles = 0;
    size_t total = 0;
    qm_tuning tuning{256, 2, 0};
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid = 0;
    std::string signature;
    // recorded on the caller's stream after every launch that reads the
    // device table, so that a re-upload (new tuning) or the final free waits
    // for the launches already queued, whatever stream they went to
    cudaEvent_t last_run = nullptr;
    bool ran = false;
};

namespace qm {

static void drop_graph(qm_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Wait for the last launch that reads the device table (any stream).
static qm_status wait_last_run(qm_batch* b)
{
    if (b->ran && b->last_run && cudaEventSynchronize(b->last_run) != cudaSuccess)
        return fail(QM_ERR_CUDA, "qm_batch: waiting for the previous run failed");
    b->ran = false;
    return QM_OK;
}

static void mark_run(qm_batch* b, cudaStream_t s)
{
    if (b->last_run && cudaEventRecord(b->last_run, s) == cudaSuccess) b->ran = true;
}

// Recompute tile prefixes for the current tuning and upload the table (after
// the launches already queued against the old table have finished).
static qm_status layout(qm_batch* b)
{
    const qm_status ws = wait_last_run(b);
    if (ws != QM_OK) return ws;
    const unsigned long long tile = (unsigned long long)b->tuning.block * b->tuning.ept;
    unsigned long long t0 = 0;
    for (auto& s : b->host) {
        s.tile0 = t0;
        t0 += (s.n + tile - 1) / tile;
    }
    b->ntiles = t0;
    if (cudaMemcpy(b->dev, b->host.data(), sizeof(DevSeg) * b->host.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return fail(QM_ERR_CUDA, "qm_batch: segment table upload failed");
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, pick_kernel(b->tuning.ept, b->tuning.estrin),
                                                  b->tuning.block, 0);
    if (bps < 1) bps = 1;
    const int sms = sm_count() > 0 ? sm_count() : 1;
    unsigned long long g = std::min<unsigned long long>(b->ntiles, (unsigned long long)sms * bps);
    b->grid = (int)std::max<unsigned long long>(g, 1);
    drop_graph(b);
    return QM_OK;
}

static std::string tune_cache_path()
{
    if (const char* p = std::getenv("QM_TUNE_CACHE")) return p;
    if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/qm_tune.txt";
    return "qm_tune.txt";
}

static bool cache_lookup(const std::string& sig, qm_tuning* t)
{
    FILE* f = std::fopen(tune_cache_path().c_str(), "r");
    if (!f) return false;
    char key[256];
    int bl, ep, es;
    bool found = false;
    while (std::fscanf(f, "%255s %d %d %d", key, &bl, &ep, &es) == 4)
        if (sig == key) {
            *t = qm_tuning{bl, ep, es};
            found = valid_tuning(*t);
        }
    std::fclose(f);
    return found;
}

static void cache_store(const std::string& sig, const qm_tuning& t)
{
    const std::string path = tune_cache_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos) {
        std::string dir = path.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') {
                const std::string part = dir.substr(0, i);
                if (!part.empty()) (void)mkdir(part.c_str(), 0755);
            }
    }
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d\n", sig.c_str(), t.block, t.ept, t.estrin);
    std::fclose(f);
}

}  // namespace qm

extern "C" qm_status qm_batch_create(const qm_segment* segs, int nseg, const qm_tuning* tuning,
                                    qm_batch** out)
{
    if (!out) return fail(QM_ERR_INVALID, "qm_batch_create: out is NULL");
    *out = nullptr;
    if (nseg <= 0 || !segs) return fail(QM_ERR_INVALID, "qm_batch_create: empty segment table");
    if (tuning && !valid_tuning(*tuning))
        return fail(QM_ERR_INVALID, "qm_batch_create: tuning (%d, %d, %d) not in the candidate set",
                    tuning->block, tuning->ept, tuning->estrin);
    std::vector<DevSeg> host(nseg);
    size_t total = 0;
    int hist[3] = {0, 0, 0};
    for (int i = 0; i < nseg; ++i) {
        const qm_segment& s = segs[i];
        DevSeg d{};
        if (s.src == QM_DIST_NORMAL && s.dst == QM_DIST_STUDENT_T) {
            if (!(s.nu > 0.0)) return fail(QM_ERR_INVALID, "qm_batch_create: segment %d: nu must be > 0", i);
            const void* tseg = nullptr;
            const double* ttail = nullptr;
            const qm_status st = t_select(s.nu, &d.t.k, &tseg, &ttail);
            if (st != QM_OK) return st;
            d.t.seg = (const ttbl::TRows*)tseg;
            d.t.tail = ttail;
            d.kind = KIND_T;
        } else if (s.src == QM_DIST_EXPONENTIAL && s.dst == QM_DIST_NORMAL) {
            d.kind = KIND_EXP;
        } else if (s.src == QM_DIST_UNIFORM && s.dst == QM_DIST_NORMAL) {
            d.kind = KIND_UNIFORM;
        } else {
            return fail(QM_ERR_INVALID, "qm_batch_create: segment %d: unsupported pair (%d -> %d)", i, s.src, s.dst);
        }
        if (s.n > 0 && (!s.in || !s.out)) return fail(QM_ERR_INVALID, "qm_batch_create: segment %d: null pointer", i);
        if (s.n > 0 && bad_overlap(s.in, s.n * 8, s.out, s.n * 8))
            return fail(QM_ERR_INVALID, "qm_batch_create: segment %d: in and out partially overlap", i);
        d.in = s.in;
        d.out = s.out;
        d.n = s.n;
        host[i] = d;
        total += s.n;
        hist[d.kind]++;
    }
    // outputs of different segments must not overlap
    std::vector<std::pair<uintptr_t, uintptr_t>> rng;
    for (auto& d : host)
        if (d.n) rng.push_back({(uintptr_t)d.out, (uintptr_t)d.out + d.n * 8});
    std::sort(rng.begin(), rng.end());
    for (size_t i = 1; i < rng.size(); ++i)
        if (rng[i].first < rng[i - 1].second)
            return fail(QM_ERR_INVALID, "qm_batch_create: output ranges of two segments overlap");
    qm_batch* b = new (std::nothrow) qm_batch;
    if (!b) return fail(QM_ERR_NOMEM, "qm_batch_create: host allocation failed");
    b->host = std::move(host);
    b->nseg = nseg;
    b->total = total;
    char sig[128];
    int lg = 0;
    while ((total >> lg) > 1) ++lg;
    std::snprintf(sig, sizeof sig, "batch:%d:%d:%d:%d:%d", nseg, lg, hist[0], hist[1], hist[2]);
    b->signature = sig;
    qm_tuning t{256, 2, 0};
    if (tuning) t = *tuning;
    else cache_lookup(b->signature, &t);
    b->tuning = t;
    if (cudaMalloc(&b->dev, sizeof(DevSeg) * nseg) != cudaSuccess) {
        delete b;
        return fail(QM_ERR_NOMEM, "qm_batch_create: device table allocation failed");
    }
    if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(b->dev);
        delete b;
        return fail(QM_ERR_CUDA, "qm_batch_create: stream creation failed");
    }
    if (cudaEventCreateWithFlags(&b->last_run, cudaEventDisableTiming) != cudaSuccess) {
        b->last_run = nullptr;
        qm_batch_destroy(b);
        return fail(QM_ERR_CUDA, "qm_batch_create: event creation failed");
    }
    const qm_status st = layout(b);
    if (st != QM_OK) {
        qm_batch_destroy(b);
        return st;
    }
    *out = b;
    return QM_OK;
}

extern "C" qm_status qm_batch_get_tuning(const qm_batch* b, qm_tuning* t)
{
    if (!b || !t) return fail(QM_ERR_INVALID, "qm_batch_get_tuning: null argument");
    *t = b->tuning;
    return QM_OK;
}

extern "C" qm_status qm_batch_set_tuning(qm_batch* b, const qm_tuning* t)
{
    if (!b || !t) return fail(QM_ERR_INVALID, "qm_batch_set_tuning: null argument");
    if (!valid_tuning(*t)) return fail(QM_ERR_INVALID, "qm_batch_set_tuning: invalid tuning");
    b->tuning = *t;
    return layout(b);
}

extern "C" qm_status qm_batch_run(qm_batch* b, void* stream)
{
    if (!b) return fail(QM_ERR_INVALID, "qm_batch_run: null batch");
    if (b->ntiles == 0) return QM_OK;
    if (!b->exec) {
        BatchKernel k = pick_kernel(b->tuning.ept, b->tuning.estrin);
        qm_status fst;
        const fxt::FxTable* fxT = (const fxt::FxTable*)fx_table_device(&fst);
        if (!fxT) return fst;
        if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(QM_ERR_CUDA, "qm_batch_run: stream capture failed to start");
        k<<<b->grid, b->tuning.block, 0, b->capture>>>(b->dev, b->nseg, b->ntiles, fxT);
        cudaError_t e = cudaStreamEndCapture(b->capture, &b->graph);
        if (e != cudaSuccess) return fail(QM_ERR_CUDA, "qm_batch_run: capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return fail(QM_ERR_CUDA, "qm_batch_run: instantiate: %s", cudaGetErrorString(e));
        }
    }
    const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(QM_ERR_CUDA, "qm_batch_run: graph launch: %s", cudaGetErrorString(e));
    mark_run(b, (cudaStream_t)stream);
    return QM_OK;
}

extern "C" qm_status qm_batch_run_separate(qm_batch* b, void* stream)
{
    if (!b) return fail(QM_ERR_INVALID, "qm_batch_run_separate: null batch");
    const int sms = sm_count() > 0 ? sm_count() : 1;
    qm_status fst;
    const fxt::FxTable* fxT = (const fxt::FxTable*)fx_table_device(&fst);
    if (!fxT) return fst;
    for (const DevSeg& s : b->host) {
        if (!s.n) continue;
        int g = (int)std::min<size_t>((s.n + 255) / 256, (size_t)sms * 8);
        k_single<<<g, 256, 0, (cudaStream_t)stream>>>(s.in, s.out, s.n, s.kind, s.t, fxT);
    }
    return check_launch("qm_batch_run_separate");
}

extern "C" qm_status qm_batch_tune(qm_batch* b, int reps, void* stream, qm_tuning* best_out)
{
    if (!b) return fail(QM_ERR_INVALID, "qm_batch_tune: null batch");
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const qm_tuning saved = b->tuning;
    qm_tuning best = saved;
    float best_ms = 1e30f;
    const int blocks[3] = {128, 256, 512}, epts[3] = {1, 2, 4};
    for (int es = 0; es <= 1; ++es)
        for (int bl : blocks)
            for (int ep : epts) {
                const qm_tuning t{bl, ep, es};
                b->tuning = t;
                if (layout(b) != QM_OK) continue;
                if (qm_batch_run(b, stream) != QM_OK) continue;     // warm-up + graph build
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps; ++r) qm_batch_run(b, stream);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= reps;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuning = best;
    const qm_status st = layout(b);
    if (st != QM_OK) return st;
    cache_store(b->signature, best);
    if (best_out) *best_out = best;
    return check_launch("qm_batch_tune");
}

extern "C" qm_status qm_batch_destroy(qm_batch* b)
{
    if (!b) return QM_OK;
    (void)wait_last_run(b);           // queued launches still read the table
    drop_graph(b);
    if (b->dev) cudaFree(b->dev);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->last_run) cudaEventDestroy(b->last_run);
    delete b;
    return QM_OK;
}
