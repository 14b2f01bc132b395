// api.cu -- the C ABI of libsam (declared in include/sam.h): handles, the
// stream-ordered device workspace, host/device argument staging, and the
// orchestration of the pattern, build, residual and apply pipelines.
//
// Batches.  K maps of order n are processed as one block-diagonal problem of
// order N = K n (see common.cuh), so every stage is one launch whatever K is.
// Patterns built together (sam_pattern_build_batched) share one
// block-diagonal store (a "pattern group"); sam_build_batched on exactly
// such a group uses it in place, any other combination is concatenated into
// a temporary group first.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

struct sam_handle_t {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sms = 1;
    uint32_t flags = 0;
    cudaMemPool_t pool = nullptr;
    int32_t *d_flag = nullptr;  // sticky device status word
    int32_t *h_flag = nullptr;  // pinned mirror
    int32_t *h_bins = nullptr;  // pinned: one map's size-class offsets [kNumBins+1] (chunked builds)
    // tracing
    int64_t launches = 0;
    bool profiling = false;
    struct Ev {
        int bin;
        cudaEvent_t a, b;
    };
    std::vector<Ev> pending;
    double lsq_ms[sam::kNumBins] = {0};
    int64_t lsq_n[sam::kNumBins] = {0};
    // FP32 tile shape per size class (sam_tune / sam_set_tile_variants)
    int variant[sam::kNumBins] = {0};
    // bin schedule (sam_tune / sam_set_bin_schedule): identity by default
    sam::BinSchedule sched = {{0, 1, 2, 3, 4, 5}};
    // the tuner's record of the last build's columns per size class
    bool record_hist = false;
    int32_t *h_hist = nullptr;  // pinned [kNumBins + 1] work-list offsets
    // refinement outcomes of the last guarded build (automatic, or a fixed
    // number of steps >= 1): columns per outcome, and a pinned mirror
    int64_t *d_refine = nullptr;
    int64_t *h_refine = nullptr;
    // factor tape (sam_set_factor_tape): the caller's device buffer
    int tape_mode = sam::kTapeOff;
    void *tape_buf = nullptr;
    int64_t tape_bytes = 0;
};

namespace {
// Builds whose map values go to a host array: at most kMaxChunks chunks of
// maps, each of about kChunkColumns columns or more (each chunk boundary
// costs the tail of a persistent launch; the last chunk's copy is exposed,
// so the last chunk is the smallest)
constexpr int kMaxChunks = 8;
constexpr int64_t kChunkColumns = 1 << 17;

// Maps [start[q], start[q+1]) form chunk q, q < count
struct MapChunks {
    int count;
    int start[kMaxChunks + 1];
};

// K maps of n columns in chunks: none (one chunk) unless the values go to
// the host; else the last chunk holds about half a share (at least one
// map) and the others split the rest evenly
MapChunks plan_chunks(int K, int64_t n, bool host_values) {
    MapChunks c;
    c.count = 1;
    c.start[0] = 0;
    c.start[1] = K;
    if (!host_values) return c;
    const int64_t want = std::min<int64_t>(std::min<int64_t>(K, kMaxChunks), std::max<int64_t>(1, (int64_t)K * n / kChunkColumns));
    if (want < 2) return c;
    const int C = (int)want;
    const int last = std::max(1, K / (2 * C));
    const int rest = K - last;
    c.count = C;
    for (int q = 0; q < C - 1; ++q) c.start[q] = (int)((int64_t)rest * q / (C - 1));
    c.start[C - 1] = rest;
    c.start[C] = K;
    return c;
}

// K patterns of order n stored as one block-diagonal pattern
struct PatternGroup {
    sam_handle h = nullptr;
    int refs = 0;
    int K = 0, n = 0;
    int32_t *jcp = nullptr, *jri = nullptr;  // CSC, rows of map k shifted by k n
    int32_t *mrp = nullptr, *mci = nullptr;  // CSR of the block-diagonal map
    int32_t *csr_pos = nullptr;              // CSC entry -> CSR position
    std::vector<int64_t> off;                // per-map nnz prefix [K+1]
    bool symmetric = false;                  // every map's pattern is structurally symmetric
    bool shared = false;                     // every map has the same pattern (built once, replicated)
};
}  // namespace

// A captured numeric rebuild (see sam_plan_create in sam.h)
struct sam_plan_t {
    sam_handle h = nullptr;
    PatternGroup *g = nullptr;     // holds one reference
    std::vector<void *> mem;       // workspace from the handle's pool
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;          // kernels per replay
};


struct sam_pattern_t {
    PatternGroup *g = nullptr;
    int k = 0;
    int n = 0;
    int64_t nnz = 0;
    int32_t *view_cp = nullptr, *view_ri = nullptr;  // local (unshifted) views, made on demand
};

namespace sam {

void *pool_alloc(sam_handle h, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMallocFromPoolAsync(&p, bytes, h->pool, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void pool_free(sam_handle h, void *p) {
    if (p) cudaFreeAsync(p, h->stream);
}
cudaStream_t handle_stream(sam_handle h) { return h->stream; }
int handle_sms(sam_handle h) { return h->sms; }
int32_t *handle_flag(sam_handle h) { return h->d_flag; }
void count_launch(sam_handle h, int n) { h->launches += n; }
int handle_variant(sam_handle h, int bin) { return h->variant[bin]; }
BinSchedule handle_schedule(sam_handle h) { return h->sched; }

void profile_begin(sam_handle h, int bin) {
    if (!h->profiling) return;
    sam_handle_t::Ev e{bin, nullptr, nullptr};
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(e.a, h->stream);
    h->pending.push_back(e);
}

void profile_end(sam_handle h, int bin) {
    if (!h->profiling || h->pending.empty() || h->pending.back().bin != bin) return;
    cudaEventRecord(h->pending.back().b, h->stream);
}

static void profile_resolve(sam_handle h) {
    for (auto &e : h->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
            h->lsq_ms[e.bin] += ms;
            h->lsq_n[e.bin] += 1;
        }
        cudaGetLastError();
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    h->pending.clear();
}

}  // namespace sam

using namespace sam;

namespace {

// Scope guard for workspace allocations of one call.
struct Scratch {
    sam_handle h;
    std::vector<void *> ptrs;
    explicit Scratch(sam_handle hh) : h(hh) {}
    template <typename T>
    T *get(size_t count) {
        void *p = pool_alloc(h, sizeof(T) * (count ? count : 1));
        if (p) ptrs.push_back(p);
        return (T *)p;
    }
    // hand the allocations to a longer-lived owner
    std::vector<void *> release() {
        std::vector<void *> out;
        out.swap(ptrs);
        return out;
    }
    ~Scratch() {
        for (void *p : ptrs) pool_free(h, p);
    }
};

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Resolves caller arrays to device pointers, staging host memory through the
// workspace; outputs are copied back by finish().
struct Stager {
    Scratch &sc;
    cudaStream_t st;
    struct Out {
        void *host;
        const void *dev;
        size_t bytes;
        size_t flushed;  // bytes already copied by flush_range
    };
    std::vector<Out> outs;
    bool failed = false;
    // host outputs copied early on a side stream (flush_early), joined back
    // into st by finish() or, on an error path, by the destructor
    cudaStream_t side = nullptr;
    cudaEvent_t ev_ready = nullptr, ev_done = nullptr;
    bool early_pending = false;
    // host inputs copied on a second side stream (in_deferred), joined into
    // st by join_inputs() before their first use
    cudaStream_t side_in = nullptr;
    cudaEvent_t ev_in_ready = nullptr, ev_in_done = nullptr;
    bool in_pending = false;
    Stager(Scratch &s, cudaStream_t stream) : sc(s), st(stream) {}
    ~Stager() {
        join();
        join_inputs();
        if (ev_ready) cudaEventDestroy(ev_ready);
        if (ev_done) cudaEventDestroy(ev_done);
        if (side) cudaStreamDestroy(side);
        if (ev_in_ready) cudaEventDestroy(ev_in_ready);
        if (ev_in_done) cudaEventDestroy(ev_in_done);
        if (side_in) cudaStreamDestroy(side_in);
    }
    // st waits for the deferred input copies
    void join_inputs() {
        if (!in_pending) return;
        cudaEventRecord(ev_in_done, side_in);
        cudaStreamWaitEvent(st, ev_in_done, 0);
        in_pending = false;
    }
    bool inputs_pending() const { return in_pending; }
    // As in(), but a host array is copied on the input side stream, so that
    // what st does next (work that does not read it) overlaps the copy; the
    // caller calls join_inputs() before st first reads it.
    template <typename T>
    const T *in_deferred(const T *p, size_t count) {
        if (!p || count == 0 || is_device_ptr(p)) return p;
        T *d = sc.get<T>(count);
        if (!d) {
            failed = true;
            return nullptr;
        }
        if (!side_in) {
            if (cudaStreamCreateWithFlags(&side_in, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_in_ready, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev_in_done, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                failed = true;
                return nullptr;
            }
        }
        // the buffer comes from st's stream-ordered pool: copy after it exists
        if (cudaEventRecord(ev_in_ready, st) != cudaSuccess || cudaStreamWaitEvent(side_in, ev_in_ready, 0) != cudaSuccess ||
            cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, side_in) != cudaSuccess) {
            failed = true;
            return nullptr;
        }
        in_pending = true;
        return d;
    }
    // st waits for the early copies (before the workspace they read is freed)
    void join() {
        if (!early_pending) return;
        cudaEventRecord(ev_done, side);
        cudaStreamWaitEvent(st, ev_done, 0);
        early_pending = false;
    }
    // The host output staged in dev is final once the work enqueued on st so
    // far completes: copy it to the host on a side stream, overlapping what st
    // does next.  Device outputs need nothing.
    cudaError_t flush_early(const void *dev) {
        for (size_t q = 0; q < outs.size(); ++q) {
            if (outs[q].dev != dev) continue;
            if (!side) {
                if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming) != cudaSuccess)
                    return cudaGetLastError();
            }
            cudaEventRecord(ev_ready, st);
            cudaStreamWaitEvent(side, ev_ready, 0);
            cudaError_t e = cudaMemcpyAsync(outs[q].host, outs[q].dev, outs[q].bytes, cudaMemcpyDeviceToHost, side);
            if (e != cudaSuccess) return e;
            early_pending = true;
            outs.erase(outs.begin() + (std::ptrdiff_t)q);
            return cudaSuccess;
        }
        return cudaSuccess;
    }
    // Bytes [off, off + bytes) of the host output staged in dev are final
    // once the work enqueued on st so far completes: copy them on the side
    // stream.  The output is dropped from the final copy once every byte has
    // been flushed this way (the ranges must not overlap).
    cudaError_t flush_range(const void *dev, size_t off, size_t bytes) {
        for (size_t q = 0; q < outs.size(); ++q) {
            if (outs[q].dev != dev) continue;
            if (off + bytes > outs[q].bytes) return cudaErrorInvalidValue;
            if (!side) {
                if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming) != cudaSuccess)
                    return cudaGetLastError();
            }
            if (bytes > 0) {
                cudaEventRecord(ev_ready, st);
                cudaStreamWaitEvent(side, ev_ready, 0);
                cudaError_t e = cudaMemcpyAsync((char *)outs[q].host + off, (const char *)outs[q].dev + off, bytes,
                                                cudaMemcpyDeviceToHost, side);
                if (e != cudaSuccess) return e;
                early_pending = true;
            }
            outs[q].flushed += bytes;
            if (outs[q].flushed == outs[q].bytes) outs.erase(outs.begin() + (std::ptrdiff_t)q);
            return cudaSuccess;
        }
        return cudaSuccess;
    }
    bool is_host_output(const void *dev) const {
        for (const auto &o : outs)
            if (o.dev == dev) return true;
        return false;
    }
    template <typename T>
    const T *in(const T *p, size_t count) {
        if (!p || count == 0 || is_device_ptr(p)) return p;
        T *d = sc.get<T>(count);
        if (!d || cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            failed = true;
            return nullptr;
        }
        return d;
    }
    template <typename T>
    T *out(T *p, size_t count) {
        if (!p || count == 0 || is_device_ptr(p)) return p;
        T *d = sc.get<T>(count);
        if (!d) {
            failed = true;
            return nullptr;
        }
        outs.push_back({(void *)p, (const void *)d, sizeof(T) * count, 0});
        any_host = true;
        return d;
    }
    // an array read and written by the call (staged both ways if on the host)
    template <typename T>
    T *inout(T *p, size_t count) {
        if (!p || count == 0 || is_device_ptr(p)) return p;
        T *d = sc.get<T>(count);
        if (!d || cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            failed = true;
            return nullptr;
        }
        outs.push_back({(void *)p, (const void *)d, sizeof(T) * count, 0});
        any_host = true;
        return d;
    }
    bool any_host = false;  // some output is a host array (the call must synchronise)
    bool has_host_outputs() const { return any_host; }
    cudaError_t finish() {
        for (auto &o : outs) {
            cudaError_t e = cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return e;
        }
        join();
        return cudaGetLastError();
    }
};

struct DevCsr {
    int n = 0;
    int64_t nnz = 0;
    const int32_t *rp = nullptr, *ci = nullptr;
    const double *v = nullptr;
};

// (an empty matrix, n = 0, has no columns to build a map for: rejected)
sam_status check_csr_arg(const sam_csr *A, bool need_val) {
    if (!A || A->n < 1 || A->nnz < 0 || A->nnz > INT32_MAX || !A->row_ptr || (A->nnz > 0 && !A->col_idx) ||
        (need_val && A->nnz > 0 && !A->val))
        return SAM_ERR_INVALID_ARG;
    return SAM_OK;
}

DevCsr stage_csr(Stager &sg, const sam_csr *A, bool with_val, bool defer_val = false) {
    DevCsr d;
    d.n = A->n;
    d.nnz = A->nnz;
    d.rp = sg.in(A->row_ptr, (size_t)A->n + 1);
    d.ci = sg.in(A->col_idx, (size_t)A->nnz);
    d.v = with_val ? (defer_val ? sg.in_deferred(A->val, (size_t)A->nnz) : sg.in(A->val, (size_t)A->nnz)) : nullptr;
    return d;
}

// Reads and clears the sticky device status (synchronises the stream).
sam_status drain_status(sam_handle h) {
    if (cudaMemcpyAsync(h->h_flag, h->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
    sam_status s = *h->h_flag;
    if (s != SAM_OK) cudaMemsetAsync(h->d_flag, 0, sizeof(int32_t), h->stream);
    return s;
}

// flag[0] = 1 when some matrix k in [1, K) has a structure (row pointers,
// column indices) different from matrix 0's; nnz equal (checked on the host).
// Thread t compares entries 4t .. 4t+3 of both arrays.
__global__ void structure_differs_kernel(int n, const CsrPtrs *mats, int64_t nnz, int32_t *flag) {
    const int k = blockIdx.y + 1;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const CsrPtrs a = mats[0], b = mats[k];
    bool diff = false;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (t + u <= n) diff = diff || a.rp[t + u] != b.rp[t + u];
        if (t + u < nnz) diff = diff || a.ci[t + u] != b.ci[t + u];
    }
    if (diff) *flag = 1;
}

// Whether every matrix of each range [b, e) of ms has the same structure as
// the range's first (exact comparison on the device).  Launched into
// flags[r] (device, zeroed by the caller); ranges whose nnz differ on the
// host are marked at once in *differ_host.
cudaError_t launch_structure_checks(sam_handle h, Scratch &sc, const std::vector<DevCsr> &ms,
                                    const std::vector<std::pair<int, int>> &ranges, int32_t *flags,
                                    std::vector<char> *differ_host) {
    differ_host->assign(ranges.size(), 0);
    for (size_t r = 0; r < ranges.size(); ++r) {
        const int b = ranges[r].first, e = ranges[r].second;
        if (e - b < 2) continue;
        bool eq = true;
        for (int k = b + 1; k < e; ++k) eq = eq && ms[k].n == ms[b].n && ms[k].nnz == ms[b].nnz;
        if (!eq) {
            (*differ_host)[r] = 1;
            continue;
        }
        std::vector<CsrPtrs> tab;
        for (int k = b; k < e; ++k) tab.push_back({ms[k].rp, ms[k].ci, nullptr});
        CsrPtrs *dtab = sc.get<CsrPtrs>(tab.size());
        if (!dtab) return cudaErrorMemoryAllocation;
        cudaMemcpyAsync(dtab, tab.data(), sizeof(CsrPtrs) * tab.size(), cudaMemcpyHostToDevice, h->stream);
        const int64_t cnt = (std::max<int64_t>((int64_t)ms[b].n + 1, ms[b].nnz) + 3) / 4;
        dim3 grid((unsigned)((cnt + 255) / 256 > 0 ? (cnt + 255) / 256 : 1), (unsigned)(e - b - 1));
        structure_differs_kernel<<<grid, 256, 0, h->stream>>>(ms[b].n, dtab, ms[b].nnz, flags + r);
        count_launch(h);
    }
    return cudaGetLastError();
}

// Validates the CSR structures of equal-order matrices on the device;
// synchronises once.  Nothing reads an unvalidated structure before this.
// same (nullable): for each range [b, e) of ms in same_ranges, whether all
// its matrices share one structure, found in the same synchronisation (with
// trusted inputs: one synchronisation for that alone).
sam_status validate_all(sam_handle h, Scratch &sc, const std::vector<DevCsr> &ms, std::vector<char> *sym = nullptr,
                        const std::vector<std::pair<int, int>> *same_ranges = nullptr,
                        std::vector<char> *same = nullptr, std::vector<int32_t> *maxrow = nullptr) {
    if (sym) sym->assign(ms.size(), 0);  // unknown (trusted inputs): treated as not symmetric
    if (maxrow) maxrow->assign(ms.size(), -1);  // unknown
    const size_t R = (same_ranges && same) ? same_ranges->size() : 0;
    if (same) same->assign(R, 0);
    if (((h->flags & SAM_FLAG_TRUSTED) || ms.empty()) && R > 0) {
        int32_t *flags = sc.get<int32_t>(R);
        if (!flags) return SAM_ERR_OOM;
        cudaMemsetAsync(flags, 0, sizeof(int32_t) * R, h->stream);
        std::vector<char> differ;
        if (launch_structure_checks(h, sc, ms, *same_ranges, flags, &differ) != cudaSuccess) return SAM_ERR_CUDA;
        std::vector<int32_t> hf(R, 0);
        cudaMemcpyAsync(hf.data(), flags, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
        for (size_t r = 0; r < R; ++r) (*same)[r] = !differ[r] && !hf[r];
        return SAM_OK;
    }
    if ((h->flags & SAM_FLAG_TRUSTED) || ms.empty()) return SAM_OK;
    const int K = (int)ms.size();
    std::vector<CsrPtrs> tab(K);
    std::vector<int64_t> nz(K);
    for (int k = 0; k < K; ++k) {
        tab[k] = {ms[k].rp, ms[k].ci, ms[k].v};
        nz[k] = ms[k].nnz;
    }
    CsrPtrs *dtab = sc.get<CsrPtrs>(K);
    int64_t *dnz = sc.get<int64_t>(K);
    // [0] status, [1 + k] matrix k not symmetric, [1 + K + r] range r not of
    // one structure, [1 + K + R + k] the longest row of matrix k
    const size_t W = (size_t)K + 1 + R + (maxrow ? (size_t)K : 0);
    int32_t *flag = sc.get<int32_t>(W);
    if (!dtab || !dnz || !flag) return SAM_ERR_OOM;
    cudaMemcpyAsync(dtab, tab.data(), sizeof(CsrPtrs) * K, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dnz, nz.data(), sizeof(int64_t) * K, cudaMemcpyHostToDevice, h->stream);
    cudaMemsetAsync(flag, 0, sizeof(int32_t) * W, h->stream);
    int32_t *asym = sym ? flag + 1 : nullptr;
    int32_t *mrow = maxrow ? flag + 1 + K + R : nullptr;
    // matrices of different order (the residual call) are validated one by one
    bool same_order = true;
    for (auto &m : ms) same_order &= (m.n == ms[0].n);
    if (same_order) {
        if (validate_csr_batch(h, K, ms[0].n, dtab, dnz, flag, asym, mrow) != cudaSuccess) return SAM_ERR_CUDA;
    } else {
        for (int k = 0; k < K; ++k)
            if (validate_csr_batch(h, 1, ms[k].n, dtab + k, dnz + k, flag, asym ? asym + k : nullptr,
                                   mrow ? mrow + k : nullptr) != cudaSuccess)
                return SAM_ERR_CUDA;
    }
    // the comparison reads rp[0..n] and ci[0..nnz) of each matrix, inside
    // the sizes the caller declared (nothing it reads is used as an index),
    // so it shares the synchronisation; its result counts only when the
    // validation passed
    std::vector<char> differ;
    if (R > 0 && launch_structure_checks(h, sc, ms, *same_ranges, flag + 1 + K, &differ) != cudaSuccess)
        return SAM_ERR_CUDA;
    std::vector<int32_t> hf(W, 0);
    cudaMemcpyAsync(hf.data(), flag, sizeof(int32_t) * W, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
    if (sym && hf[0] == 0)
        for (int k = 0; k < K; ++k) (*sym)[k] = hf[(size_t)k + 1] == 0;
    if (maxrow && hf[0] == 0)
        for (int k = 0; k < K; ++k) (*maxrow)[k] = hf[(size_t)K + 1 + R + k];
    if (hf[0] == 0)
        for (size_t r = 0; r < R; ++r) (*same)[r] = !differ[r] && !hf[(size_t)K + 1 + r];
    return hf[0] ? (sam_status)hf[0] : SAM_OK;
}

__global__ void scatter_inverse_kernel(int64_t nnz, const int32_t *perm, int32_t *pos) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) pos[perm[p]] = (int32_t)p;
}

__global__ void gather_strided_kernel(int K, int n, const int32_t *jcp, int64_t *off) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= K) off[k] = jcp[(int64_t)k * n];
}

void group_release(PatternGroup *g) {
    if (!g || --g->refs > 0) return;
    sam_handle h = g->h;
    pool_free(h, g->jcp);
    pool_free(h, g->jri);
    pool_free(h, g->mrp);
    pool_free(h, g->mci);
    pool_free(h, g->csr_pos);
    delete g;
}

// Completes a group from its block-diagonal CSC pattern (takes ownership of
// jcp / jri, which must come from the handle's pool): per-map offsets, the
// CSR structure of the map and the CSC -> CSR positions.
sam_status group_finish(sam_handle h, int K, int n, int32_t *jcp, int32_t *jri, int64_t nnz, PatternGroup **out,
                        bool symmetric = false) {
    PatternGroup *g = new (std::nothrow) PatternGroup;
    if (!g) return SAM_ERR_OOM;
    g->h = h;
    g->refs = 1;
    g->K = K;
    g->n = n;
    g->jcp = jcp;
    g->jri = jri;
    const int64_t N = (int64_t)K * n;
    g->mrp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)N + 1));
    g->mci = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    g->csr_pos = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    int32_t *perm = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    int64_t *doff = (int64_t *)pool_alloc(h, sizeof(int64_t) * ((size_t)K + 1));
    auto fail = [&](sam_status s) {
        pool_free(h, perm);
        pool_free(h, doff);
        group_release(g);
        return s;
    };
    if (!g->mrp || !g->mci || !g->csr_pos || !perm || !doff) return fail(SAM_ERR_OOM);
    g->symmetric = symmetric;
    if (symmetric) {
        // a symmetric pattern is its own transpose: the map's CSR structure is
        // the CSC structure, and CSC entry p sits at its mirror's position
        if (csr_to_csc(h, (int)N, nnz, jcp, jri, nullptr, g->mrp, g->mci, nullptr, nullptr, true) != cudaSuccess ||
            mirror_positions(h, (int)N, jcp, jri, g->csr_pos) != cudaSuccess)
            return fail(SAM_ERR_CUDA);
    } else {
        // the CSC of the map read as the CSR of its transpose; transposing it
        // gives the CSR of the map, with perm[p] = CSC entry of CSR position p
        if (csr_to_csc(h, (int)N, nnz, jcp, jri, nullptr, g->mrp, g->mci, nullptr, perm) != cudaSuccess)
            return fail(SAM_ERR_CUDA);
        if (nnz > 0) {
            scatter_inverse_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, h->stream>>>(nnz, perm, g->csr_pos);
            count_launch(h);
        }
    }
    g->off.resize((size_t)K + 1);
    if (K == 1) {  // one map: its offsets are known without a readback
        g->off[0] = 0;
        g->off[1] = nnz;
    } else {
        gather_strided_kernel<<<(K + 1 + 127) / 128, 128, 0, h->stream>>>(K, n, jcp, doff);
        count_launch(h);
        if (cudaMemcpyAsync(g->off.data(), doff, sizeof(int64_t) * ((size_t)K + 1), cudaMemcpyDeviceToHost,
                            h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return fail(SAM_ERR_CUDA);
    }
    pool_free(h, perm);
    pool_free(h, doff);
    *out = g;
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

// dst[k n + t] = src[t] + k step for t < n, k < K; dst[K n] = K step
__global__ void replicate_offsets_kernel(int K, int n, const int32_t *src, int32_t step, int32_t *dst) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (t < n) dst[(int64_t)k * n + t] = src[t] + k * step;
    if (k == K - 1 && t == 0) dst[(int64_t)K * n] = K * step;
}

// dst[k m + e] = src[e] + k shift for e < m, k < K
__global__ void replicate_shifted_kernel(int64_t m, const int32_t *src, int32_t shift, int32_t *dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (e < m) dst[(int64_t)k * m + e] = src[e] + k * shift;
}

// the same four entries per thread with 16-byte accesses (m a multiple of 4,
// 16-byte aligned arrays)
__global__ void replicate_shifted4_kernel(int64_t m4, const int4 *src, int32_t shift, int4 *dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (e < m4) {
        int4 v = src[e];
        const int32_t d = k * shift;
        v.x += d;
        v.y += d;
        v.z += d;
        v.w += d;
        dst[(int64_t)k * m4 + e] = v;
    }
}

void replicate_shifted(cudaStream_t st, int K, int64_t m, const int32_t *src, int32_t shift, int32_t *dst) {
    const bool vec = m % 4 == 0 && ((uintptr_t)src % 16) == 0 && ((uintptr_t)dst % 16) == 0;
    const int64_t cnt = vec ? m / 4 : m;
    const dim3 grid((unsigned)((cnt + 255) / 256 > 0 ? (cnt + 255) / 256 : 1), (unsigned)K);
    if (vec)
        replicate_shifted4_kernel<<<grid, 256, 0, st>>>(cnt, (const int4 *)src, shift, (int4 *)dst);
    else
        replicate_shifted_kernel<<<grid, 256, 0, st>>>(m, src, shift, dst);
}

// a[k n + t] = a[t] for 1 <= k < K (the per-column results of map 0)
template <typename T>
__global__ void replicate_cols_kernel(int64_t n, T *a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y + 1;
    if (t < n) a[(int64_t)k * n + t] = a[t];
}

// Work list of K maps that share one structure, from map 0's (work0 over its
// n columns, offsets off0[kNumBins + 1]): the maps interleaved column by
// column, work[K t + k] = work0[t] + k n, off[c] = K off0[c], so that the
// same column of every map is solved side by side (one block reads map 0's
// metadata for all of them)
__global__ void expand_work_kernel(int K, MapChunks ch, int n, const int32_t *work0, const int32_t *off0, int32_t *work,
                                   int32_t *off) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (t < off0[kNumBins]) {
        int b = 0;
        while (t >= off0[b + 1]) ++b;
        const int64_t c = off0[b + 1] - off0[b], tl = t - off0[b];
        // maps in chunks: a chunk's items are contiguous within the
        // class, its maps interleaved column by column
        int q = 0;
        while (q + 1 < ch.count && k >= ch.start[q + 1]) ++q;
        const int k0 = ch.start[q], wq = ch.start[q + 1] - k0;
        work[(int64_t)K * off0[b] + (int64_t)k0 * c + wq * tl + (k - k0)] = work0[t] + k * n;
    }
    if (t <= kNumBins && k == 0) off[t] = K * off0[t];
}

cudaError_t interleaved_work_list(sam_handle h, Scratch &sc, int K, int n, const uint8_t *bin, int32_t *work,
                                  int32_t *bin_off, const MapChunks *chunks = nullptr,
                                  const int32_t **off0_out = nullptr) {
    int32_t *work0 = sc.get<int32_t>((size_t)n), *off0 = sc.get<int32_t>(kNumBins + 1);
    if (!work0 || !off0) return cudaErrorMemoryAllocation;
    cudaError_t e = build_work_list(h, n, bin, work0, off0);
    if (e != cudaSuccess) return e;
    const int64_t cnt = std::max<int64_t>(n, kNumBins + 1);
    dim3 grid((unsigned)((cnt + 255) / 256), (unsigned)K);
    const MapChunks ch = chunks ? *chunks : plan_chunks(K, n, false);
    expand_work_kernel<<<grid, 256, 0, h->stream>>>(K, ch, n, work0, off0, work, bin_off);
    count_launch(h);
    if (off0_out) *off0_out = off0;
    return cudaGetLastError();
}

template <typename T>
cudaError_t replicate_cols(sam_handle h, int K, int64_t n, T *a) {
    if (K < 2 || n == 0 || !a) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)(K - 1));
    replicate_cols_kernel<T><<<grid, 256, 0, h->stream>>>(n, a);
    count_launch(h);
    return cudaGetLastError();
}

// A group of K maps that all have the pattern of g1 (a one-map group): its
// CSC pattern, map CSR structure and CSC -> CSR positions replicated with
// each map's offsets.  g1 is released.
sam_status group_replicate(sam_handle h, PatternGroup *g1, int K, PatternGroup **out) {
    const int n = g1->n;
    const int64_t m = g1->off[1];
    const int64_t N = (int64_t)K * n, tot = (int64_t)K * m;
    if (N > INT32_MAX - 1 || tot > INT32_MAX) {
        group_release(g1);
        return SAM_ERR_INVALID_ARG;
    }
    PatternGroup *g = new (std::nothrow) PatternGroup;
    if (!g) {
        group_release(g1);
        return SAM_ERR_OOM;
    }
    g->h = h;
    g->refs = 1;
    g->K = K;
    g->n = n;
    g->symmetric = g1->symmetric;
    g->shared = true;
    g->jcp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)N + 1));
    g->jri = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(tot ? tot : 1));
    g->mrp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)N + 1));
    g->mci = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(tot ? tot : 1));
    g->csr_pos = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(tot ? tot : 1));
    if (!g->jcp || !g->jri || !g->mrp || !g->mci || !g->csr_pos) {
        group_release(g);
        group_release(g1);
        return SAM_ERR_OOM;
    }
    const dim3 gn((unsigned)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1), (unsigned)K);
    replicate_offsets_kernel<<<gn, 256, 0, h->stream>>>(K, n, g1->jcp, (int32_t)m, g->jcp);
    replicate_offsets_kernel<<<gn, 256, 0, h->stream>>>(K, n, g1->mrp, (int32_t)m, g->mrp);
    replicate_shifted(h->stream, K, m, g1->jri, n, g->jri);
    replicate_shifted(h->stream, K, m, g1->mci, n, g->mci);
    replicate_shifted(h->stream, K, m, g1->csr_pos, (int32_t)m, g->csr_pos);
    count_launch(h, 5);
    g->off.resize((size_t)K + 1);
    for (int k = 0; k <= K; ++k) g->off[k] = (int64_t)k * m;
    group_release(g1);  // stream-ordered frees: the copies above read g1 first
    *out = g;
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

sam_status make_patterns(PatternGroup *g, sam_pattern *out) {
    for (int k = 0; k < g->K; ++k) {
        sam_pattern S = new (std::nothrow) sam_pattern_t;
        if (!S) {
            for (int q = 0; q < k; ++q) sam_pattern_destroy(out[q]);
            return SAM_ERR_OOM;
        }
        S->g = g;
        S->k = k;
        S->n = g->n;
        S->nnz = g->off[k + 1] - g->off[k];
        if (k > 0) g->refs++;
        out[k] = S;
    }
    return SAM_OK;
}

__global__ void rebase_view_kernel(int n, int k, const int32_t *jcp, const int32_t *jri, int64_t base, int64_t nnz,
                                   int32_t *cp, int32_t *ri) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t shift = (int64_t)k * n;
    if (t <= n) cp[t] = (int32_t)(jcp[shift + t] - base);
    if (t < nnz) ri[t] = (int32_t)(jri[base + t] - shift);
}

// Concatenate member patterns of arbitrary groups into a temporary group.
__global__ void concat_pattern_kernel(int n, int k, const int32_t *src_cp, const int32_t *src_ri, int64_t src_base,
                                      int src_k, int64_t dst_base, int32_t *dst_cp, int32_t *dst_ri, int64_t nnz,
                                      int last) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t sshift = (int64_t)src_k * n, dshift = (int64_t)k * n;
    if (t < n || (last && t == n)) dst_cp[dshift + t] = (int32_t)(src_cp[sshift + t] - src_base + dst_base);
    if (t < nnz) dst_ri[dst_base + t] = (int32_t)(src_ri[src_base + t] - sshift + dshift);
}

sam_status group_for(sam_handle h, int K, const sam_pattern *S, PatternGroup **g_out, bool *temp) {
    PatternGroup *g0 = S[0]->g;
    bool direct = g0->K == K;
    for (int k = 0; k < K && direct; ++k) direct = (S[k]->g == g0 && S[k]->k == k);
    if (direct) {
        *g_out = g0;
        *temp = false;
        return SAM_OK;
    }
    const int n = S[0]->n;
    int64_t tot = 0;
    for (int k = 0; k < K; ++k) tot += S[k]->nnz;
    if (tot > INT32_MAX) return SAM_ERR_INVALID_ARG;
    const int64_t N = (int64_t)K * n;
    int32_t *jcp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)N + 1));
    int32_t *jri = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(tot ? tot : 1));
    if (!jcp || !jri) {
        pool_free(h, jcp);
        pool_free(h, jri);
        return SAM_ERR_OOM;
    }
    int64_t base = 0;
    for (int k = 0; k < K; ++k) {
        PatternGroup *g = S[k]->g;
        const int64_t cnt = (n + 1 > S[k]->nnz) ? n + 1 : S[k]->nnz;
        concat_pattern_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, h->stream>>>(
            n, k, g->jcp, g->jri, g->off[S[k]->k], S[k]->k, base, jcp, jri, S[k]->nnz, k == K - 1);
        count_launch(h);
        base += S[k]->nnz;
    }
    *temp = true;
    bool sym = true;
    for (int k = 0; k < K; ++k) sym = sym && S[k]->g->symmetric;
    return group_finish(h, K, n, jcp, jri, tot, g_out, sym);
}

}  // namespace

namespace {
// one line per tuned problem family:
//   <device name with '_' for blanks> <SMs> <K> <n> <nnz(S) total> <precision> <steps> v0 .. v4
std::string tune_key(sam_handle h, int K, int n, int64_t nnz, int precision, int steps) {
    cudaDeviceProp p;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&p, h->device) == cudaSuccess) name = p.name;
    cudaGetLastError();
    for (char &c : name)
        if (c == ' ' || c == '\t') c = '_';
    char buf[160];
    snprintf(buf, sizeof(buf), " %d %d %d %lld %d %d", h->sms, K, n, (long long)nnz, precision, steps);
    return name + buf;
}

// A cache line: the key, then kNumBins tile variants and kNumBins entries of
// the bin schedule.
bool tune_lookup(const char *path, const std::string &key, int *v, int *to) {
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        const size_t kl = key.size();
        if (strncmp(line, key.c_str(), kl) != 0 || line[kl] != ' ') continue;
        int t[2 * kNumBins];
        const char *q = line + kl;
        bool ok = true;
        for (int b = 0; b < 2 * kNumBins && ok; ++b) {
            int used = 0;
            ok = sscanf(q, "%d%n", &t[b], &used) == 1;
            q += used;
        }
        if (!ok) continue;
        for (int b = 0; b < kNumBins; ++b) {
            ok = ok && t[b] >= 0 && t[b] < kTileVariants[b];
            const int d = t[kNumBins + b];
            ok = ok && (b == kBinBig ? d == kBinBig : (d >= b && d < kRegBins));
        }
        if (!ok) continue;
        for (int b = 0; b < kNumBins; ++b) {
            v[b] = t[b];
            to[b] = t[kNumBins + b];
        }
        found = true;  // the last matching line wins
    }
    fclose(f);
    return found;
}
}  // namespace

extern "C" {

void sam_limits(int32_t *max_rows, int32_t *max_cols) {
    if (max_rows) *max_rows = kBigICap;
    if (max_cols) *max_cols = kBigJCap;
}

sam_status sam_size_classes(int32_t *max_rows, int32_t *max_cols, int32_t *max_entries, int32_t *max_tile,
                            int32_t *variants, int count) {
    // the register tiles' capacities (lsq.cu, the shadow kernel's table) and the large class
    static const int32_t rows[kNumBins] = {14, 26, 40, 52, 64, kBigICap};
    static const int32_t cols[kNumBins] = {5, 9, 23, 27, 27, kBigJCap};
    if (count != kNumBins) return SAM_ERR_INVALID_ARG;
    for (int b = 0; b < kNumBins; ++b) {
        if (max_rows) max_rows[b] = rows[b];
        if (max_cols) max_cols[b] = cols[b];
        if (max_entries) max_entries[b] = b == kBinBig ? kBigLCap : 8 * rows[b];
        if (max_tile) max_tile[b] = b == kBinBig ? kBigTileDoubles : rows[b] * (cols[b] + 1);
        if (variants) variants[b] = kTileVariants[b];
    }
    return SAM_OK;
}

const char *sam_status_string(sam_status s) {
    switch (s) {
        case SAM_OK: return "ok";
        case SAM_ERR_INVALID_ARG: return "invalid argument";
        case SAM_ERR_BAD_CSR: return "malformed CSR/CSC structure";
        case SAM_ERR_RANK_DEFICIENT: return "rank-deficient column least-squares problem";
        case SAM_ERR_NONFINITE: return "non-finite value in a column solve";
        case SAM_ERR_CUDA: return "CUDA runtime error";
        case SAM_ERR_OOM: return "out of device memory";
        case SAM_ERR_TIMEOUT: return "timed out";
        case SAM_ERR_UNSUPPORTED: return "column exceeds the kernel size limits";
        default: return "unknown status";
    }
}

sam_status sam_create(sam_handle *out, void *cuda_stream) {
    if (!out) return SAM_ERR_INVALID_ARG;
    *out = nullptr;
    sam_handle h = new (std::nothrow) sam_handle_t;
    if (!h) return SAM_ERR_OOM;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return SAM_ERR_CUDA;
    }
    h->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = h->device;
    if (cudaMemPoolCreate(&h->pool, &props) != cudaSuccess) {
        delete h;
        return SAM_ERR_CUDA;
    }
    uint64_t thr = UINT64_MAX;  // keep freed blocks for reuse
    cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    if (cudaMalloc(&h->d_flag, sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&h->d_refine, sizeof(int64_t) * (kAutoSteps + 1)) != cudaSuccess ||
        cudaMallocHost(&h->h_flag, sizeof(int32_t) * (2 + kNumBins)) != cudaSuccess ||
        cudaMallocHost(&h->h_refine, sizeof(int64_t) * (kAutoSteps + 1)) != cudaSuccess ||
        cudaMallocHost(&h->h_hist, sizeof(int32_t) * (kNumBins + 1)) != cudaSuccess) {
        cudaGetLastError();
        if (h->d_flag) cudaFree(h->d_flag);
        if (h->d_refine) cudaFree(h->d_refine);
        if (h->h_flag) cudaFreeHost(h->h_flag);
        if (h->h_refine) cudaFreeHost(h->h_refine);
        cudaMemPoolDestroy(h->pool);
        delete h;
        return SAM_ERR_OOM;
    }
    cudaMemset(h->d_flag, 0, sizeof(int32_t));
    cudaMemset(h->d_refine, 0, sizeof(int64_t) * (kAutoSteps + 1));
    *h->h_flag = 0;
    h->h_bins = h->h_flag + 1;
    *out = h;
    return SAM_OK;
}

sam_status sam_destroy(sam_handle h) {
    if (!h) return SAM_ERR_INVALID_ARG;
    cudaStreamSynchronize(h->stream);
    h->profiling = false;
    profile_resolve(h);
    cudaFree(h->d_flag);
    cudaFree(h->d_refine);
    cudaFreeHost(h->h_flag);
    cudaFreeHost(h->h_refine);
    cudaFreeHost(h->h_hist);
    cudaMemPoolDestroy(h->pool);
    delete h;
    return SAM_OK;
}

sam_status sam_set_stream(sam_handle h, void *cuda_stream) {
    if (!h) return SAM_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    return SAM_OK;
}

sam_status sam_set_flags(sam_handle h, uint32_t flags) {
    if (!h) return SAM_ERR_INVALID_ARG;
    h->flags = flags;
    return SAM_OK;
}

sam_status sam_sync(sam_handle h) {
    if (!h) return SAM_ERR_INVALID_ARG;
    return drain_status(h);
}

sam_status sam_pattern_build_batched(sam_handle h, int K, const sam_csr *A, int level, sam_pattern *out) {
    if (!h || K < 1 || !A || !out || level < 0 || level > 3) return SAM_ERR_INVALID_ARG;
    int64_t tot = 0;
    for (int k = 0; k < K; ++k) {
        out[k] = nullptr;
        if (check_csr_arg(&A[k], false) != SAM_OK || A[k].n != A[0].n) return SAM_ERR_INVALID_ARG;
        tot += A[k].nnz;
    }
    const int n = A[0].n;
    const int64_t N = (int64_t)K * n;
    if (N > INT32_MAX - 1 || tot > INT32_MAX) return SAM_ERR_INVALID_ARG;
    cudaStream_t st = h->stream;
    Scratch sc(h);
    Stager sg(sc, st);
    std::vector<DevCsr> d(K);
    // host structures: map 0's now, the others on the input side stream; a
    // batch of one structure needs map 0's alone for its pattern, which is
    // built while the others copy (and dropped if they turn out to differ)
    d[0] = stage_csr(sg, &A[0], false);
    for (int k = 1; k < K; ++k) {
        d[k].n = A[k].n;
        d[k].nnz = A[k].nnz;
        d[k].rp = sg.in_deferred(A[k].row_ptr, (size_t)A[k].n + 1);
        d[k].ci = sg.in_deferred(A[k].col_idx, (size_t)A[k].nnz);
    }
    if (sg.failed) return SAM_ERR_OOM;
    // map 0's pattern (level-L CSC), built once
    struct Map0Pattern {
        sam_handle h;
        int32_t *jcp = nullptr, *jri = nullptr;
        int64_t nnz = 0;
        bool built = false;
        ~Map0Pattern() {  // released unless handed to a pattern group
            pool_free(h, jcp);
            pool_free(h, jri);
        }
    } p0{h};
    // (a structurally symmetric matrix's columns are as long as its rows, so
    // its longest row bounds the pattern's candidate lists: maxcol)
    auto build_map0 = [&](bool sym0, int maxcol) -> sam_status {
        int32_t *kcp = sc.get<int32_t>((size_t)n + 1), *kri = sc.get<int32_t>((size_t)d[0].nnz);
        if (!kcp || !kri) return SAM_ERR_OOM;
        if (csr_to_csc(h, n, d[0].nnz, d[0].rp, d[0].ci, nullptr, kcp, kri, nullptr, nullptr, sym0) != cudaSuccess)
            return SAM_ERR_CUDA;
        p0.built = true;
        return level_pattern(h, n, kcp, kri, d[0].nnz, level, &p0.jcp, &p0.jri, &p0.nnz, sym0 ? maxcol : -1);
    };
    sam_status s;
    bool sym0 = false;
    if (sg.inputs_pending()) {
        std::vector<char> sv0;
        std::vector<int32_t> mr0;
        s = validate_all(h, sc, {d[0]}, &sv0, nullptr, nullptr, &mr0);
        if (s != SAM_OK) return s;
        sym0 = sv0[0] != 0;
        if ((s = build_map0(sym0, mr0[0])) != SAM_OK) return s;
        sg.join_inputs();
    }
    std::vector<char> symv, same;
    std::vector<int32_t> mrow;
    const std::vector<std::pair<int, int>> whole{{0, K}};
    s = validate_all(h, sc, d, &symv, K > 1 ? &whole : nullptr, &same, &mrow);
    if (s != SAM_OK) return s;
    bool sym = true;
    int maxrow = 0;
    for (char c : symv) sym = sym && c;
    for (int32_t m : mrow) maxrow = m < 0 ? -1 : (maxrow < 0 ? -1 : std::max(maxrow, (int)m));
    if (K > 1 && same[0]) {
        // one structure for the whole sequence (the paper's setting, Sec. 2):
        // the pattern of map 0, replicated for every map
        if (!p0.built && (s = build_map0(sym, mrow[0])) != SAM_OK) return s;
        int32_t *jcp = p0.jcp, *jri = p0.jri;
        const int64_t nnz = p0.nnz;
        p0.jcp = p0.jri = nullptr;  // owned by the group from here
        PatternGroup *g1 = nullptr, *g = nullptr;
        s = group_finish(h, 1, n, jcp, jri, nnz, &g1, sym);
        if (s != SAM_OK) return s;
        s = group_replicate(h, g1, K, &g);
        if (s != SAM_OK) return s;
        s = make_patterns(g, out);
        if (s != SAM_OK) {
            group_release(g);
            return s;
        }
        // the status word was read with the pattern's size (level_pattern)
        return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
    }
    // block-diagonal structure of the batch, then its CSC
    std::vector<CsrPtrs> tab(K);
    std::vector<int64_t> off(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        tab[k] = {d[k].rp, d[k].ci, nullptr};
        off[k + 1] = off[k] + d[k].nnz;
    }
    CsrPtrs *dtab = sc.get<CsrPtrs>(K);
    int64_t *doff = sc.get<int64_t>(K + 1);
    int32_t *brp = sc.get<int32_t>((size_t)N + 1), *bci = sc.get<int32_t>((size_t)tot);
    int32_t *kcp = sc.get<int32_t>((size_t)N + 1), *kri = sc.get<int32_t>((size_t)tot);
    if (!dtab || !doff || !brp || !bci || !kcp || !kri) return SAM_ERR_OOM;
    cudaMemcpyAsync(dtab, tab.data(), sizeof(CsrPtrs) * K, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st);
    if (concat_block_diag(h, K, n, dtab, doff, brp, bci, nullptr) != cudaSuccess) return SAM_ERR_CUDA;
    if (csr_to_csc(h, (int)N, tot, brp, bci, nullptr, kcp, kri, nullptr, nullptr, sym) != cudaSuccess)
        return SAM_ERR_CUDA;
    int32_t *jcp = nullptr, *jri = nullptr;
    int64_t nnz = 0;
    s = level_pattern(h, (int)N, kcp, kri, tot, level, &jcp, &jri, &nnz, sym ? maxrow : -1);
    if (s != SAM_OK) return s;
    PatternGroup *g = nullptr;
    // level-L patterns of a structurally symmetric matrix are symmetric
    s = group_finish(h, K, n, jcp, jri, nnz, &g, sym);
    if (s != SAM_OK) return s;
    s = make_patterns(g, out);
    if (s != SAM_OK) {
        group_release(g);
        return s;
    }
    // the status word was read with the pattern's size (level_pattern)
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

sam_status sam_pattern_build(sam_handle h, const sam_csr *A_k, int level, sam_pattern *out) {
    return sam_pattern_build_batched(h, 1, A_k, level, out);
}

sam_status sam_pattern_from_csc(sam_handle h, int32_t n, int64_t nnz, const int32_t *colptr, const int32_t *rowidx,
                                sam_pattern *out) {
    if (!h || !out || n < 1 || nnz < n || nnz > INT32_MAX || !colptr || !rowidx) return SAM_ERR_INVALID_ARG;
    *out = nullptr;
    int32_t *jcp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
    int32_t *jri = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    if (!jcp || !jri) {
        pool_free(h, jcp);
        pool_free(h, jri);
        return SAM_ERR_OOM;
    }
    cudaMemcpyAsync(jcp, colptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDefault, h->stream);
    cudaMemcpyAsync(jri, rowidx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDefault, h->stream);
    // the pattern is a CSC structure: validate it as the CSR of its transpose,
    // plus the requirement that every column is nonempty (checked on the host
    // copy of the column pointers)
    std::vector<int32_t> hcp((size_t)n + 1);
    cudaMemcpyAsync(hcp.data(), jcp, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost, h->stream);
    bool user_sym = false;
    {
        Scratch sc(h);
        DevCsr d;
        d.n = n;
        d.nnz = nnz;
        d.rp = jcp;
        d.ci = jri;
        uint32_t saved = h->flags;
        h->flags &= ~(uint32_t)SAM_FLAG_TRUSTED;  // a pattern is always validated
        std::vector<char> symv;
        sam_status s = validate_all(h, sc, {d}, &symv);
        h->flags = saved;
        user_sym = s == SAM_OK && symv[0];
        bool nonempty = true;
        for (int j = 0; j < n && s == SAM_OK; ++j) nonempty &= hcp[(size_t)j + 1] > hcp[j];
        if (s == SAM_OK && !nonempty) s = SAM_ERR_BAD_CSR;
        if (s != SAM_OK) {
            pool_free(h, jcp);
            pool_free(h, jri);
            return s;
        }
    }
    PatternGroup *g = nullptr;
    sam_status s = group_finish(h, 1, n, jcp, jri, nnz, &g, user_sym);
    if (s != SAM_OK) return s;
    return make_patterns(g, out);
}

sam_status sam_pattern_get(sam_pattern S, int32_t *n, int64_t *nnz, const int32_t **colptr, const int32_t **rowidx) {
    if (!S) return SAM_ERR_INVALID_ARG;
    if (n) *n = S->n;
    if (nnz) *nnz = S->nnz;
    PatternGroup *g = S->g;
    if (colptr || rowidx) {
        if (g->K == 1) {
            if (colptr) *colptr = g->jcp;
            if (rowidx) *rowidx = g->jri;
            return SAM_OK;
        }
        sam_handle h = g->h;
        if (!S->view_cp) {
            S->view_cp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)S->n + 1));
            S->view_ri = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(S->nnz ? S->nnz : 1));
            if (!S->view_cp || !S->view_ri) return SAM_ERR_OOM;
            const int64_t cnt = (S->n + 1 > S->nnz) ? S->n + 1 : S->nnz;
            rebase_view_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, h->stream>>>(
                S->n, S->k, g->jcp, g->jri, g->off[S->k], S->nnz, S->view_cp, S->view_ri);
            count_launch(h);
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
        }
        if (colptr) *colptr = S->view_cp;
        if (rowidx) *rowidx = S->view_ri;
    }
    return SAM_OK;
}

sam_status sam_pattern_destroy(sam_pattern S) {
    if (!S) return SAM_ERR_INVALID_ARG;
    sam_handle h = S->g->h;
    pool_free(h, S->view_cp);
    pool_free(h, S->view_ri);
    group_release(S->g);
    delete S;
    return SAM_OK;
}

}  // extern "C"

namespace {

// K matrices of order n as one block-diagonal CSC of order K n (with the
// CSC -> CSR permutation when perm != nullptr); K = 1 skips the copy.
sam_status block_diag_csc(sam_handle h, Scratch &sc, const std::vector<DevCsr> &ms, int n, int32_t **cp,
                          int32_t **ri, double **cv, int32_t **perm, int64_t *total, Scratch *tmp_sc = nullptr,
                          bool symmetric = false, bool values_later = false) {
    Scratch &tmp = tmp_sc ? *tmp_sc : sc;  // the concatenated copy lives only until the transpose
    const int K = (int)ms.size();
    const int64_t N = (int64_t)K * n;
    int64_t tot = 0;
    std::vector<CsrPtrs> tab(K);
    std::vector<int64_t> off(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        tab[k] = {ms[k].rp, ms[k].ci, values_later ? nullptr : ms[k].v};
        off[k + 1] = off[k] + ms[k].nnz;
    }
    tot = off[K];
    *total = tot;
    *cp = sc.get<int32_t>((size_t)N + 1);
    *ri = sc.get<int32_t>((size_t)tot);
    *cv = sc.get<double>((size_t)tot);
    if (perm) *perm = sc.get<int32_t>((size_t)tot);
    if (!*cp || !*ri || !*cv || (perm && !*perm)) return SAM_ERR_OOM;
    const int32_t *rp = ms[0].rp, *ci = ms[0].ci;
    const double *v = ms[0].v;
    if (K > 1) {
        CsrPtrs *dtab = tmp.get<CsrPtrs>(K);
        int64_t *doff = tmp.get<int64_t>(K + 1);
        int32_t *brp = tmp.get<int32_t>((size_t)N + 1), *bci = tmp.get<int32_t>((size_t)tot);
        double *bv = values_later ? nullptr : tmp.get<double>((size_t)tot);
        if (!dtab || !doff || !brp || !bci || (!values_later && !bv)) return SAM_ERR_OOM;
        cudaMemcpyAsync(dtab, tab.data(), sizeof(CsrPtrs) * K, cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, h->stream);
        if (concat_block_diag(h, K, n, dtab, doff, brp, bci, bv) != cudaSuccess) return SAM_ERR_CUDA;
        rp = brp;
        ci = bci;
        v = bv;
    }
    if (csr_to_csc(h, (int)N, tot, rp, ci, values_later ? nullptr : v, *cp, *ri, values_later ? nullptr : *cv,
                   perm ? *perm : nullptr, symmetric) != cudaSuccess)
        return SAM_ERR_CUDA;
    return SAM_OK;
}

// Values of K sources of one structure in the CSC order of the first: map
// k's go to positions k nnz + q through the first's CSC -> CSR positions.
sam_status shared_csc_values(sam_handle h, Scratch &sc, const std::vector<DevCsr> &ms, const int32_t *perm,
                             double *cv) {
    const int K = (int)ms.size();
    std::vector<const double *> vals(K);
    for (int k = 0; k < K; ++k) vals[k] = ms[k].v;
    const double **dvals = sc.get<const double *>(K);
    if (!dvals) return SAM_ERR_OOM;
    cudaMemcpyAsync(dvals, vals.data(), sizeof(const double *) * K, cudaMemcpyHostToDevice, h->stream);
    return gather_values_shared(h, ms[0].nnz, K, dvals, perm, cv) == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

// The values of a block_diag_csc made with values_later (and its perm): map
// k's columns hold exactly its own entries, positions [off_k, off_k+1) of
// the CSC, and perm gives each one's position in the concatenated CSR.
sam_status block_diag_values(sam_handle h, Scratch &sc, const std::vector<DevCsr> &ms, const int32_t *perm,
                             double *cv) {
    const int K = (int)ms.size();
    std::vector<const double *> vals(K);
    std::vector<int64_t> off(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        vals[k] = ms[k].v;
        off[k + 1] = off[k] + ms[k].nnz;
    }
    if (off[K] == 0) return SAM_OK;
    const double **dvals = sc.get<const double *>(K);
    int64_t *doff = sc.get<int64_t>(K + 1);
    if (!dvals || !doff) return SAM_ERR_OOM;
    cudaMemcpyAsync(dvals, vals.data(), sizeof(const double *) * K, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, h->stream);
    return gather_values(h, off[K], K, doff, dvals, perm, cv, nullptr) == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

// K maps of order n against NT = 1 shared target or NT = K targets (one per map)
// Factor tape of a batch on pattern group g: slot offsets (device, [N+1])
// and the bytes they need, read back (synchronises the handle's stream).
sam_status tape_layout(sam_handle h, Scratch &sc, const PatternGroup *g, int64_t N, int precision, int64_t **off,
                       int64_t *bytes) {
    int64_t *sizes = sc.get<int64_t>((size_t)(N > 0 ? N : 1));
    *off = sc.get<int64_t>((size_t)N + 1);
    if (!sizes || !*off) return SAM_ERR_OOM;
    int64_t tot = 0;
    if (tape_offsets(h, N, g->jcp, sizes, *off) != cudaSuccess ||
        cudaMemcpyAsync(&tot, *off + N, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return SAM_ERR_CUDA;
    *bytes = tot * (precision == SAM_FP64 ? (int64_t)sizeof(double) : (int64_t)sizeof(float));
    return SAM_OK;
}

// the handle's tape, if it is in `mode`, for a batch on group g: sets the
// launch arguments, or fails if the caller's buffer is too small
sam_status tape_args(sam_handle h, Scratch &sc, const PatternGroup *g, int64_t N, int precision, int mode,
                     LsqArgs &a) {
    if (h->tape_mode != mode) return SAM_OK;
    int64_t *off = nullptr, bytes = 0;
    sam_status s = tape_layout(h, sc, g, N, precision, &off, &bytes);
    if (s != SAM_OK) return s;
    if (bytes > h->tape_bytes) return SAM_ERR_INVALID_ARG;
    a.fac = h->tape_buf;
    a.fac_off = off;
    a.fac_mode = mode;
    return SAM_OK;
}

sam_status build_impl(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, int NT, const sam_pattern *S,
                      int precision, int refine_steps, const int64_t *M_offsets, int32_t *M_row_ptr,
                      int32_t *M_col_idx, double *M_val, int32_t *col_status, double *res2, double *fro) {
    if (!h || K < 1 || !A_k || !A_0 || !S || !M_offsets || !M_row_ptr || !M_col_idx || !M_val)
        return SAM_ERR_INVALID_ARG;
    if (precision != SAM_FP64 && precision != SAM_FP32_REFINE) return SAM_ERR_INVALID_ARG;
    if (refine_steps < SAM_REFINE_AUTO || refine_steps > 4) return SAM_ERR_INVALID_ARG;
    const int n = A_0[0].n;
    int64_t ktot = 0, ztot = 0;
    for (int t = 0; t < NT; ++t) {
        if (check_csr_arg(&A_0[t], true) != SAM_OK || A_0[t].n != n) return SAM_ERR_INVALID_ARG;
        ztot += A_0[t].nnz;
    }
    if (M_offsets[0] != 0) return SAM_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (check_csr_arg(&A_k[k], true) != SAM_OK || A_k[k].n != n || !S[k] || S[k]->n != n)
            return SAM_ERR_INVALID_ARG;
        if (M_offsets[k + 1] - M_offsets[k] != S[k]->nnz) return SAM_ERR_INVALID_ARG;
        ktot += A_k[k].nnz;
    }
    const int64_t N = (int64_t)K * n;
    const int64_t total_nnz = M_offsets[K];
    if (N > INT32_MAX - 1 || ktot > INT32_MAX || ztot > INT32_MAX || total_nnz > INT32_MAX)
        return SAM_ERR_INVALID_ARG;
    cudaStream_t st = h->stream;
    Scratch sc(h);
    Stager sg(sc, st);
    // host values are copied on a side stream while the validation and the
    // structure work (which read the structures alone) run on st
    std::vector<DevCsr> zs(NT);
    for (int t = 0; t < NT; ++t) zs[t] = stage_csr(sg, &A_0[t], true, true);
    std::vector<DevCsr> ak(K);
    for (int k = 0; k < K; ++k) ak[k] = stage_csr(sg, &A_k[k], true, true);
    const bool late = sg.inputs_pending();
    int32_t *d_rp = sg.out(M_row_ptr, (size_t)K * ((size_t)n + 1));
    int32_t *d_ci = sg.out(M_col_idx, (size_t)total_nnz);
    double *d_v = sg.out(M_val, (size_t)total_nnz);
    int32_t *d_st = col_status ? sg.out(col_status, (size_t)N) : nullptr;
    double *d_r2 = res2 ? sg.out(res2, (size_t)N) : nullptr;
    if (sg.failed) return SAM_ERR_OOM;
    bool ksym = true, zsym = true;  // structurally symmetric sources / targets
    bool one_structure = false;     // every source, every target: one structure each
    {
        std::vector<DevCsr> all(ak);
        all.insert(all.end(), zs.begin(), zs.end());
        std::vector<char> symv, same;
        const std::vector<std::pair<int, int>> ranges{{0, K}, {K, K + NT}};
        sam_status s = validate_all(h, sc, all, &symv, K > 1 ? &ranges : nullptr, &same);
        if (s != SAM_OK) return s;
        for (size_t q = 0; q < symv.size(); ++q) (q < ak.size() ? ksym : zsym) &= symv[q] != 0;
        one_structure = K > 1 && same[0] && same[1];
    }
    PatternGroup *g = nullptr;
    bool temp = false;
    {
        sam_status s = group_for(h, K, S, &g, &temp);
        if (s != SAM_OK) return s;
    }
    struct GroupGuard {
        PatternGroup *g;
        bool temp;
        ~GroupGuard() {
            if (temp) group_release(g);
        }
    } guard{g, temp};
    // shadow rows, local rows and size classes depend on the structures
    // alone: with one source structure, one target structure and one
    // pattern for all maps, map 0's are computed and shared
    const bool shared = one_structure && g->shared;
    const int NS = shared ? n : (int)N;  // columns whose shadow data is computed
    // target(s) and sources as CSC with values
    int32_t *zcp = nullptr, *zri = nullptr, *kcp = nullptr, *kri = nullptr;
    double *zcv = nullptr, *kcv = nullptr;
    int32_t *zperm = nullptr, *kperm = nullptr;  // with late values: CSC -> CSR positions
    int64_t zn = 0, kn = 0;
    sam_status s = block_diag_csc(h, sc, zs, n, &zcp, &zri, &zcv, late ? &zperm : nullptr, &zn, nullptr, zsym, late);
    if (s != SAM_OK) return s;
    // one structure: the kernels read map 0's CSC structure for every map, so
    // only map 0 is transposed and each map's values are gathered into map
    // 0's CSC order through its CSC -> CSR positions (map k at k nnz_0)
    const bool one_csc = shared && K > 1;
    if (one_csc) {
        const std::vector<DevCsr> first{ak[0]};
        double *unused = nullptr;
        int64_t kn0 = 0;
        s = block_diag_csc(h, sc, first, n, &kcp, &kri, &unused, &kperm, &kn0, nullptr, ksym, true);
        if (s != SAM_OK) return s;
        kn = (int64_t)K * kn0;
        kcv = sc.get<double>((size_t)kn);
        if (!kcv) return SAM_ERR_OOM;
        if (!late && (s = shared_csc_values(h, sc, ak, kperm, kcv)) != SAM_OK) return s;
    } else {
        s = block_diag_csc(h, sc, ak, n, &kcp, &kri, &kcv, late ? &kperm : nullptr, &kn, nullptr, ksym, late);
        if (s != SAM_OK) return s;
    }
    int32_t *ish = sc.get<int32_t>((size_t)N * kICap), *icnt = sc.get<int32_t>((size_t)N);
    uint8_t *bin = sc.get<uint8_t>((size_t)N);
    int32_t *work = sc.get<int32_t>((size_t)N);
    int32_t *bin_off = sc.get<int32_t>(kNumBins + 1);
    if (!d_st) d_st = sc.get<int32_t>((size_t)N);
    if (!d_r2) d_r2 = sc.get<double>((size_t)N);
    uint8_t *lrow = sc.get<uint8_t>((size_t)N * kLCap);
    uint8_t *zloc = sc.get<uint8_t>((size_t)N * kZCap);
    if (!ish || !icnt || !bin || !work || !bin_off || !d_st || !d_r2 || !lrow || !zloc)
        return SAM_ERR_OOM;
    // shadow rows, size classes, work list
    ShadowTarget tg;
    tg.zcp = zcp;
    tg.zri = zri;
    tg.zbig = NT > 1 ? 1 : 0;
    tg.n = n;
    tg.zloc = zloc;
    if (shadow_and_bins(h, NS, kcp, kri, g->jcp, g->jri, ish, icnt, bin, d_st, nullptr, lrow, tg) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (shared && (replicate_cols(h, K, n, icnt) != cudaSuccess || replicate_cols(h, K, n, bin) != cudaSuccess ||
                   replicate_cols(h, K, n, d_st) != cudaSuccess))
        return SAM_ERR_CUDA;
    // Map values going to a host array: the solves of the large size classes
    // run in chunks of maps, and each chunk's values are copied to the host
    // while the next chunk is solved (one structure only, where every map has
    // the same columns per class; the automatic mode re-solves columns after
    // all chunks and is left whole)
    // automatic refinement, or a fixed number of steps >= 1: columns that
    // miss the accuracy target are re-solved in FP64 after the solves
    const bool autoref = precision == SAM_FP32_REFINE && refine_steps < 0;
    const bool guarded = precision == SAM_FP32_REFINE && refine_steps != 0;
    const MapChunks chunks = plan_chunks(K, n, shared && !autoref && sg.is_host_output(d_v));
    const bool chunked = chunks.count > 1;
    cudaEvent_t ev_bins = nullptr;
    struct EventGuard {
        cudaEvent_t &e;
        ~EventGuard() {
            if (e) cudaEventDestroy(e);
        }
    } ev_guard{ev_bins};
    const int32_t *off0 = nullptr;
    if ((shared ? interleaved_work_list(h, sc, K, n, bin, work, bin_off, &chunks, &off0)
                : build_work_list(h, (int)N, bin, work, bin_off)) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (h->record_hist &&
        cudaMemcpyAsync(h->h_hist, bin_off, sizeof(int32_t) * (kNumBins + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (chunked && (cudaEventCreateWithFlags(&ev_bins, cudaEventDisableTiming) != cudaSuccess ||
                    cudaMemcpyAsync(h->h_bins, off0, sizeof(int32_t) * (kNumBins + 1), cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess ||
                    cudaEventRecord(ev_bins, st) != cudaSuccess))
        return SAM_ERR_CUDA;
    cudaMemsetAsync(d_v, 0, sizeof(double) * (size_t)total_nnz, st);
    cudaMemsetAsync(d_r2, 0, sizeof(double) * (size_t)N, st);
    // CSR structure of every map (it depends on the patterns alone): written
    // before the solves, so that a copy to host outputs overlaps them
    if (split_map_structure(h, K, n, g->mrp, g->mci, d_rp, d_ci) != cudaSuccess ||
        sg.flush_early(d_rp) != cudaSuccess || sg.flush_early(d_ci) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (late) {
        sg.join_inputs();
        if ((s = block_diag_values(h, sc, zs, zperm, zcv)) != SAM_OK) return s;
        if ((s = one_csc ? shared_csc_values(h, sc, ak, kperm, kcv) : block_diag_values(h, sc, ak, kperm, kcv)) != SAM_OK)
            return s;
    }
    float *kcv32 = nullptr, *zcv32 = nullptr;
    if (precision == SAM_FP32_REFINE) {
        kcv32 = sc.get<float>((size_t)kn);
        zcv32 = sc.get<float>((size_t)zn);
        if (!kcv32 || !zcv32) return SAM_ERR_OOM;
        if (round_to_f32(h, kn, kcv, kcv32) != cudaSuccess || round_to_f32(h, zn, zcv, zcv32) != cudaSuccess)
            return SAM_ERR_CUDA;
    }
    LsqArgs a;
    memset(&a, 0, sizeof(a));
    a.kcv32 = kcv32;
    a.zcv32 = zcv32;
    a.n = n;
    a.kcp = kcp;
    a.kri = kri;
    a.kcv = kcv;
    a.jcp = g->jcp;
    a.jri = g->jri;
    a.ish = ish;
    a.icnt = icnt;
    a.lrow = lrow;
    a.zcp = zcp;
    a.zri = zri;
    a.zcv = zcv;
    a.zbig = NT > 1 ? 1 : 0;
    a.zloc = zloc;
    a.shadow_shared = shared ? 1 : 0;
    a.map_nnz_src = ak[0].nnz;
    a.map_nnz_pat = g->off[1] - g->off[0];
    a.csr_pos = g->csr_pos;
    a.mval = d_v;
    a.colres = d_r2;
    a.colstat = d_st;
    a.work = work;
    a.bin_off = bin_off;
    a.refine_steps = refine_steps;
    if ((s = tape_args(h, sc, g, N, precision, kTapeRecord, a)) != SAM_OK) return s;
    int32_t *work2 = nullptr, *bin_off2 = nullptr;
    RedoLists redo;
    if (guarded) {
        a.refine_used = sc.get<uint8_t>((size_t)N);
        work2 = sc.get<int32_t>((size_t)N);
        bin_off2 = sc.get<int32_t>(2);
        if (!a.refine_used || !work2 || !bin_off2) return SAM_ERR_OOM;
        cudaMemsetAsync(a.refine_used, 0, (size_t)N, st);
    }
    if (autoref) {
        // columns that ask for a second step are solved again by a launch of their own
        redo.bin = bin;
        redo.bins2 = sc.get<uint8_t>((size_t)N);
        redo.work = sc.get<int32_t>((size_t)N);
        redo.bin_off = sc.get<int32_t>(kNumBins + 1);
        redo.ws = sc.get<int32_t>(2 * kNumBins);
        if (!redo.bins2 || !redo.work || !redo.bin_off || !redo.ws) return SAM_ERR_OOM;
    }
    if (!chunked) {
        if (launch_lsq(h, precision, a) != cudaSuccess) return SAM_ERR_CUDA;
    } else {
        // one map's columns per class (the work list is read back while the
        // launches above run); classes holding a quarter of the columns or
        // more are chunked, the others go first over all maps
        if (cudaEventSynchronize(ev_bins) != cudaSuccess) return SAM_ERR_CUDA;
        int cnt[kNumBins];
        bool big[kNumBins];
        for (int b = 0; b < kNumBins; ++b) {
            cnt[b] = h->h_bins[b + 1] - h->h_bins[b];
            big[b] = (int64_t)cnt[b] * 4 >= n;
            if (!big[b] && launch_lsq_bin(h, precision, a, b) != cudaSuccess) return SAM_ERR_CUDA;
        }
        for (int q = 0; q < chunks.count; ++q) {
            const int k0 = chunks.start[q], k1 = chunks.start[q + 1];
            for (int b = 0; b < kNumBins; ++b) {
                if (!big[b]) continue;
                LsqArgs ac = a;
                ac.item_lo = k0 * cnt[b];
                ac.item_hi = k1 * cnt[b];
                if (launch_lsq_bin(h, precision, ac, b) != cudaSuccess) return SAM_ERR_CUDA;
            }
            if (sg.flush_range(d_v, sizeof(double) * (size_t)M_offsets[k0],
                               sizeof(double) * (size_t)(M_offsets[k1] - M_offsets[k0])) != cudaSuccess)
                return SAM_ERR_CUDA;
        }
    }
    if (guarded && launch_refine_fallback(h, a, (int)N, work2, bin_off2, h->d_refine, redo) != cudaSuccess)
        return SAM_ERR_CUDA;
    // chunked host values were copied before the re-solves: their count comes
    // back with the final synchronisation, and re-solved columns are copied again
    if (chunked && guarded &&
        cudaMemcpyAsync(h->h_refine, h->d_refine, sizeof(int64_t) * (kAutoSteps + 1), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
        return SAM_ERR_CUDA;
    auto recopy_values = [&]() -> sam_status {
        if (!(chunked && guarded) || h->h_refine[kAutoSteps] == 0) return SAM_OK;
        if (cudaMemcpyAsync(M_val, d_v, sizeof(double) * (size_t)total_nnz, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SAM_ERR_CUDA;
        return SAM_OK;
    };
    if (status_reduce(h, d_st, N, h->d_flag) != cudaSuccess) return SAM_ERR_CUDA;
    double *fro_dev = nullptr;
    if (fro) {
        fro_dev = sc.get<double>((size_t)K);
        if (!fro_dev) return SAM_ERR_OOM;
        if (segmented_sum_f64(h, d_r2, K, n, fro_dev, false) != cudaSuccess) return SAM_ERR_CUDA;
    }
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    if (fro) {
        std::vector<double> f2(K);
        if (cudaMemcpyAsync(f2.data(), fro_dev, sizeof(double) * K, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SAM_ERR_CUDA;
        s = drain_status(h);
        for (int k = 0; k < K; ++k) fro[k] = sqrt(f2[k]);
        const sam_status r = recopy_values();
        return s != SAM_OK ? s : r;
    }
    if (sg.has_host_outputs()) {
        s = drain_status(h);
        const sam_status r = recopy_values();
        return s != SAM_OK ? s : r;
    }
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

}  // namespace

extern "C" {

sam_status sam_build_batched(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, const sam_pattern *S,
                             int precision, int refine_steps, const int64_t *M_offsets, int32_t *M_row_ptr,
                             int32_t *M_col_idx, double *M_val, int32_t *col_status, double *res2, double *fro) {
    return build_impl(h, K, A_k, A_0, 1, S, precision, refine_steps, M_offsets, M_row_ptr, M_col_idx, M_val,
                      col_status, res2, fro);
}

sam_status sam_build_multi(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, const sam_pattern *S,
                           int precision, int refine_steps, const int64_t *M_offsets, int32_t *M_row_ptr,
                           int32_t *M_col_idx, double *M_val, int32_t *col_status, double *res2, double *fro) {
    return build_impl(h, K, A_k, A_0, K, S, precision, refine_steps, M_offsets, M_row_ptr, M_col_idx, M_val,
                      col_status, res2, fro);
}

sam_status sam_build(sam_handle h, const sam_csr *A_k, const sam_csr *A_0, sam_pattern S, int precision,
                     int refine_steps, int32_t *M_row_ptr, int32_t *M_col_idx, double *M_val, int32_t *col_status,
                     double *res2) {
    if (!S) return SAM_ERR_INVALID_ARG;
    int64_t off[2] = {0, S->nnz};
    return sam_build_batched(h, 1, A_k, A_0, &S, precision, refine_steps, off, M_row_ptr, M_col_idx, M_val,
                             col_status, res2, nullptr);
}

sam_status sam_sparsify(sam_handle h, const sam_csr *A, int mode, double param, int32_t *S_row_ptr,
                        int32_t *S_col_idx, double *S_val, int64_t *S_nnz) {
    if (!h || !A || !S_row_ptr || !S_col_idx || !S_nnz) return SAM_ERR_INVALID_ARG;
    if (check_csr_arg(A, true) != SAM_OK) return SAM_ERR_INVALID_ARG;
    if (mode < SAM_SPARSIFY_GLOBAL || mode > SAM_SPARSIFY_LFIL || !std::isfinite(param)) return SAM_ERR_INVALID_ARG;
    if (mode == SAM_SPARSIFY_TAU && (param < 0.0 || param > 1.0)) return SAM_ERR_INVALID_ARG;
    if (mode == SAM_SPARSIFY_LFIL && param < 0.0) return SAM_ERR_INVALID_ARG;
    const int n = A->n;
    cudaStream_t st = h->stream;
    Scratch sc(h);
    Stager sg(sc, st);
    DevCsr a = stage_csr(sg, A, true);
    int32_t *d_rp = sg.out(S_row_ptr, (size_t)n + 1);
    int32_t *d_ci = sg.out(S_col_idx, (size_t)a.nnz);
    double *d_v = S_val ? sg.out(S_val, (size_t)a.nnz) : nullptr;
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, sc, {a});
    if (s != SAM_OK) return s;
    uint8_t *keep = sc.get<uint8_t>((size_t)a.nnz);
    int32_t *cnt = sc.get<int32_t>((size_t)n + 1);
    if (!keep || !cnt) return SAM_ERR_OOM;
    if (mode != SAM_SPARSIFY_LFIL && n > 0 && a.nnz > 0) {
        // row-wise decisions: the table form, which fuses the counts
        const CsrPtrs tab{a.rp, a.ci, a.v};
        const int64_t off[2] = {0, a.nnz};
        CsrPtrs *dtab = sc.get<CsrPtrs>(1);
        int64_t *doff = sc.get<int64_t>(2), *koff = sc.get<int64_t>(2);
        int32_t *orp = sc.get<int32_t>((size_t)n + 1);
        if (!dtab || !doff || !koff || !orp) return SAM_ERR_OOM;
        cudaMemcpyAsync(dtab, &tab, sizeof(CsrPtrs), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(doff, off, sizeof(off), cudaMemcpyHostToDevice, st);
        if (sparsify_rows_batched(h, 1, n, dtab, doff, a.nnz, mode == SAM_SPARSIFY_GLOBAL ? 0 : 1, param, keep, cnt,
                                  orp, d_rp, d_ci, d_v, koff) != cudaSuccess)
            return SAM_ERR_CUDA;
    } else if (sparsify_keep(h, n, a.nnz, a.rp, a.ci, a.v, mode, param, keep) != cudaSuccess ||
               compact_kept(h, n, a.rp, a.ci, a.v, keep, cnt, d_rp, d_ci, d_v) != cudaSuccess) {
        return SAM_ERR_CUDA;
    }
    int32_t kept = 0;
    if (cudaMemcpyAsync(&kept, d_rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    s = drain_status(h);
    *S_nnz = kept;
    return s;
}

sam_status sam_sparsify_batched(sam_handle h, int K, const sam_csr *A, int mode, double param, int32_t *S_row_ptr,
                                int32_t *S_col_idx, double *S_val, int64_t *S_offsets) {
    if (!h || K < 1 || !A || !S_row_ptr || !S_col_idx || !S_offsets) return SAM_ERR_INVALID_ARG;
    if (mode < SAM_SPARSIFY_GLOBAL || mode > SAM_SPARSIFY_LFIL || !std::isfinite(param)) return SAM_ERR_INVALID_ARG;
    if (mode == SAM_SPARSIFY_TAU && (param < 0.0 || param > 1.0)) return SAM_ERR_INVALID_ARG;
    if (mode == SAM_SPARSIFY_LFIL && param < 0.0) return SAM_ERR_INVALID_ARG;
    int64_t tot = 0;
    for (int k = 0; k < K; ++k) {
        if (check_csr_arg(&A[k], true) != SAM_OK || A[k].n != A[0].n) return SAM_ERR_INVALID_ARG;
        tot += A[k].nnz;
    }
    const int n = A[0].n;
    const int64_t N = (int64_t)K * n;
    if (N > INT32_MAX - 1 || tot > INT32_MAX) return SAM_ERR_INVALID_ARG;
    cudaStream_t st = h->stream;
    Scratch sc(h);
    Stager sg(sc, st);
    std::vector<DevCsr> d(K);
    for (int k = 0; k < K; ++k) d[k] = stage_csr(sg, &A[k], true);
    int32_t *d_rp = sg.out(S_row_ptr, (size_t)K * (n + 1));
    int32_t *d_ci = sg.out(S_col_idx, (size_t)tot);
    double *d_v = S_val ? sg.out(S_val, (size_t)tot) : nullptr;
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, sc, d);
    if (s != SAM_OK) return s;
    // the sparsifications act within a column, a row, or on a pair of
    // diagonal entries of the same matrix, so the block-diagonal
    // concatenation of the batch sparsifies map by map in one pass
    std::vector<CsrPtrs> tab(K);
    std::vector<int64_t> off(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        tab[k] = {d[k].rp, d[k].ci, d[k].v};
        off[k + 1] = off[k] + d[k].nnz;
    }
    CsrPtrs *dtab = sc.get<CsrPtrs>(K);
    int64_t *doff = sc.get<int64_t>(K + 1);
    if (mode != SAM_SPARSIFY_LFIL && n > 0 && tot > 0) {
        // row-wise decisions: every map read in place through the table
        uint8_t *keep = sc.get<uint8_t>((size_t)tot);
        int32_t *cnt = sc.get<int32_t>((size_t)N + 1), *orp = sc.get<int32_t>((size_t)N + 1);
        int64_t *koff = sc.get<int64_t>((size_t)K + 1);
        if (!dtab || !doff || !keep || !cnt || !orp || !koff) return SAM_ERR_OOM;
        cudaMemcpyAsync(dtab, tab.data(), sizeof(CsrPtrs) * K, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st);
        if (sparsify_rows_batched(h, K, n, dtab, doff, tot, mode == SAM_SPARSIFY_GLOBAL ? 0 : 1, param, keep, cnt,
                                  orp, d_rp, d_ci, d_v, koff) != cudaSuccess)
            return SAM_ERR_CUDA;
        std::vector<int64_t> hoff((size_t)K + 1, 0);
        if (cudaMemcpyAsync(hoff.data(), koff, sizeof(int64_t) * (K + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SAM_ERR_CUDA;
        if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
        s = drain_status(h);
        for (int k = 0; k <= K; ++k) S_offsets[k] = hoff[k];
        return s;
    }
    int32_t *brp = sc.get<int32_t>((size_t)N + 1), *bci = sc.get<int32_t>((size_t)tot);
    double *bv = sc.get<double>((size_t)tot);
    uint8_t *keep = sc.get<uint8_t>((size_t)tot);
    int32_t *cnt = sc.get<int32_t>((size_t)N + 1);
    int32_t *orp = sc.get<int32_t>((size_t)N + 1), *oci = sc.get<int32_t>((size_t)tot);
    int64_t *koff = sc.get<int64_t>((size_t)K + 1);
    if (!dtab || !doff || !brp || !bci || !bv || !keep || !cnt || !orp || !oci || !koff) return SAM_ERR_OOM;
    cudaMemcpyAsync(dtab, tab.data(), sizeof(CsrPtrs) * K, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st);
    if (concat_block_diag(h, K, n, dtab, doff, brp, bci, bv) != cudaSuccess ||
        sparsify_keep(h, (int)N, tot, brp, bci, bv, mode, param, keep) != cudaSuccess ||
        compact_kept(h, (int)N, brp, bci, bv, keep, cnt, orp, oci, d_v) != cudaSuccess ||
        split_map_structure(h, K, n, orp, oci, d_rp, d_ci) != cudaSuccess)
        return SAM_ERR_CUDA;
    gather_strided_kernel<<<(K + 1 + 127) / 128, 128, 0, st>>>(K, n, orp, koff);
    count_launch(h);
    if (cudaGetLastError() != cudaSuccess) return SAM_ERR_CUDA;
    std::vector<int64_t> hoff((size_t)K + 1, 0);
    if (cudaMemcpyAsync(hoff.data(), koff, sizeof(int64_t) * (K + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    s = drain_status(h);
    for (int k = 0; k <= K; ++k) S_offsets[k] = hoff[k];
    return s;
}

sam_status sam_residual(sam_handle h, const sam_csr *A_k, const sam_csr *M_k, const sam_csr *A_0, double *fro,
                        double *rel) {
    if (!h || check_csr_arg(A_k, true) || check_csr_arg(M_k, true) || check_csr_arg(A_0, true))
        return SAM_ERR_INVALID_ARG;
    const int n = A_k->n;
    if (M_k->n != n || A_0->n != n) return SAM_ERR_INVALID_ARG;
    Scratch sc(h);
    Stager sg(sc, h->stream);
    DevCsr a = stage_csr(sg, A_k, true), m = stage_csr(sg, M_k, true), z = stage_csr(sg, A_0, true);
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, sc, {a, m, z});
    if (s != SAM_OK) return s;
    double *rr = sc.get<double>((size_t)n), *out = sc.get<double>(2);
    if (!rr || !out) return SAM_ERR_OOM;
    if (residual_rows(h, n, a.rp, a.ci, a.v, m.rp, m.ci, m.v, z.rp, z.ci, z.v, rr, h->d_flag) != cudaSuccess ||
        sum_f64(h, rr, n, out, false) != cudaSuccess || sum_f64(h, z.v, z.nnz, out + 1, true) != cudaSuccess)
        return SAM_ERR_CUDA;
    double hv[2] = {0, 0};
    if (cudaMemcpyAsync(hv, out, sizeof(hv), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return SAM_ERR_CUDA;
    s = drain_status(h);
    if (fro) *fro = sqrt(hv[0]);
    if (rel) *rel = hv[1] > 0 ? sqrt(hv[0]) / sqrt(hv[1]) : 0.0;
    return s;
}

sam_status sam_apply(sam_handle h, const sam_csr *M_k, const double *x, double *y) {
    if (!h || check_csr_arg(M_k, true) || !x || !y) return SAM_ERR_INVALID_ARG;
    const int n = M_k->n;
    Scratch sc(h);
    Stager sg(sc, h->stream);
    DevCsr m = stage_csr(sg, M_k, true);
    const double *dx = sg.in(x, (size_t)n);
    double *dy = sg.out(y, (size_t)n);
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, sc, {m});
    if (s != SAM_OK) return s;
    if (csr_spmv(h, n, m.rp, m.ci, m.v, dx, dy) != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.has_host_outputs()) return drain_status(h);
    return SAM_OK;
}

sam_status sam_apply_grad(sam_handle h, const sam_csr *M_k, const double *x, const double *dy, double *dM_val) {
    if (!h || check_csr_arg(M_k, false) || !x || !dy || !dM_val) return SAM_ERR_INVALID_ARG;
    const int n = M_k->n;
    Scratch sc(h);
    Stager sg(sc, h->stream);
    DevCsr m = stage_csr(sg, M_k, false);
    const double *dx = sg.in(x, (size_t)n);
    const double *ddy = sg.in(dy, (size_t)n);
    double *dg = sg.out(dM_val, (size_t)M_k->nnz);
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, sc, {m});
    if (s != SAM_OK) return s;
    if (csr_outer_on_pattern(h, n, m.rp, m.ci, ddy, dx, dg) != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.has_host_outputs()) return drain_status(h);
    return SAM_OK;
}

sam_status sam_gmres(sam_handle h, const sam_csr *A, const sam_csr *M, const sam_csr *P_0, const double *b, double *x,
                     int restart, int maxiter, double rtol, int32_t *iters, double *relres, double *history) {
    if (!h || check_csr_arg(A, true) || !b || !x) return SAM_ERR_INVALID_ARG;
    if (restart < 1 || restart > SAM_GMRES_MAX_RESTART || maxiter < 0 || !std::isfinite(rtol) || rtol < 0.0)
        return SAM_ERR_INVALID_ARG;
    const int n = A->n;
    if ((M && (check_csr_arg(M, true) || M->n != n)) || (P_0 && (check_csr_arg(P_0, true) || P_0->n != n)))
        return SAM_ERR_INVALID_ARG;
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    if (n == 0) return SAM_OK;
    Scratch sc(h);
    Stager sg(sc, h->stream);
    std::vector<DevCsr> all;
    all.push_back(stage_csr(sg, A, true));
    DevCsr dm, dp;
    if (M) all.push_back(dm = stage_csr(sg, M, true));
    if (P_0) all.push_back(dp = stage_csr(sg, P_0, true));
    const double *db = sg.in(b, (size_t)n);
    double *dx = sg.inout(x, (size_t)n);
    double *dh = (history && maxiter > 0) ? sg.out(history, (size_t)maxiter) : nullptr;
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, sc, all);
    if (s != SAM_OK) return s;
    KryOp a{all[0].nnz, all[0].rp, all[0].ci, all[0].v}, m, p;
    if (M) m = KryOp{dm.nnz, dm.rp, dm.ci, dm.v};
    if (P_0) p = KryOp{dp.nnz, dp.rp, dp.ci, dp.v};
    int32_t its = 0;
    double rel = 0.0;
    s = gmres_solve(h, 1, n, &a, M ? &m : nullptr, p, db, dx, restart, maxiter, rtol, dh, &its, &rel, nullptr);
    if (iters) *iters = its;
    if (relres) *relres = rel;
    if (s != SAM_OK) return s;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    return drain_status(h);
}

sam_status sam_gmres_batched(sam_handle h, int K, const sam_csr *A, const sam_csr *M, const sam_csr *P_0,
                             const double *b, double *x, int restart, int maxiter, double rtol, int32_t *iters,
                             double *relres, double *history) {
    if (!h || K < 1 || !A || !b || !x) return SAM_ERR_INVALID_ARG;
    if (restart < 1 || restart > SAM_GMRES_MAX_RESTART || maxiter < 0 || !std::isfinite(rtol) || rtol < 0.0)
        return SAM_ERR_INVALID_ARG;
    const int n = A[0].n;
    for (int k = 0; k < K; ++k) {
        if (check_csr_arg(&A[k], true) || A[k].n != n) return SAM_ERR_INVALID_ARG;
        if (M && (check_csr_arg(&M[k], true) || M[k].n != n)) return SAM_ERR_INVALID_ARG;
    }
    if (P_0 && (check_csr_arg(P_0, true) || P_0->n != n)) return SAM_ERR_INVALID_ARG;
    const int64_t N = (int64_t)K * n;
    if (N > INT32_MAX) return SAM_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (iters) iters[k] = 0;
        if (relres) relres[k] = 0.0;
    }
    if (n == 0) return SAM_OK;
    Scratch sc(h);
    Stager sg(sc, h->stream);
    std::vector<DevCsr> all;
    for (int k = 0; k < K; ++k) all.push_back(stage_csr(sg, &A[k], true));
    if (M)
        for (int k = 0; k < K; ++k) all.push_back(stage_csr(sg, &M[k], true));
    if (P_0) all.push_back(stage_csr(sg, P_0, true));
    const double *db = sg.in(b, (size_t)N);
    double *dx = sg.inout(x, (size_t)N);
    double *dh = (history && maxiter > 0) ? sg.out(history, (size_t)K * maxiter) : nullptr;
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, sc, all);
    if (s != SAM_OK) return s;
    std::vector<KryOp> a(K), m(M ? K : 0);
    for (int k = 0; k < K; ++k) {
        a[k] = KryOp{all[k].nnz, all[k].rp, all[k].ci, all[k].v};
        if (M) m[k] = KryOp{all[K + k].nnz, all[K + k].rp, all[K + k].ci, all[K + k].v};
    }
    KryOp p;
    if (P_0) {
        const DevCsr &d = all.back();
        p = KryOp{d.nnz, d.rp, d.ci, d.v};
    }
    std::vector<int32_t> its((size_t)K, 0);
    std::vector<double> rel((size_t)K, 0.0);
    s = gmres_solve(h, K, n, a.data(), M ? m.data() : nullptr, p, db, dx, restart, maxiter, rtol, dh, its.data(),
                    rel.data(), nullptr);
    for (int k = 0; k < K; ++k) {
        if (iters) iters[k] = its[k];
        if (relres) relres[k] = rel[k];
    }
    if (s != SAM_OK) return s;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    return drain_status(h);
}

}  // extern "C"

namespace {

// adjoint of K maps, each against its own target
sam_status backward_impl(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, const sam_pattern *S,
                         int precision, int refine_steps, const int64_t *M_offsets, const double *M_val,
                         const double *dM_val, double resid_weight, double *dA_k_val, double *dA_0_val,
                         double *dM_resid) {
    if (!h || K < 1 || !A_k || !A_0 || !S || !M_offsets || !M_val || !dA_k_val || !dA_0_val)
        return SAM_ERR_INVALID_ARG;
    if (precision != SAM_FP64 && precision != SAM_FP32_REFINE) return SAM_ERR_INVALID_ARG;
    if (refine_steps < SAM_REFINE_AUTO || refine_steps > 4 || !std::isfinite(resid_weight)) return SAM_ERR_INVALID_ARG;
    if (refine_steps < 0) refine_steps = kAutoSteps;  // lambda: the automatic mode's largest step count
    const int n = A_0[0].n;
    int64_t ktot = 0, ztot = 0;
    if (M_offsets[0] != 0) return SAM_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (check_csr_arg(&A_k[k], true) != SAM_OK || check_csr_arg(&A_0[k], true) != SAM_OK) return SAM_ERR_INVALID_ARG;
        if (A_k[k].n != n || A_0[k].n != n || !S[k] || S[k]->n != n) return SAM_ERR_INVALID_ARG;
        if (M_offsets[k + 1] - M_offsets[k] != S[k]->nnz) return SAM_ERR_INVALID_ARG;
        ktot += A_k[k].nnz;
        ztot += A_0[k].nnz;
    }
    const int64_t N = (int64_t)K * n;
    const int64_t mtot = M_offsets[K];
    if (N > INT32_MAX - 1 || ktot > INT32_MAX || ztot > INT32_MAX || mtot > INT32_MAX) return SAM_ERR_INVALID_ARG;
    cudaStream_t st = h->stream;
    Scratch sc(h);
    Stager sg(sc, st);
    std::vector<DevCsr> ak(K), zs(K);
    for (int k = 0; k < K; ++k) {
        ak[k] = stage_csr(sg, &A_k[k], true);
        zs[k] = stage_csr(sg, &A_0[k], true);
    }
    const double *d_m = sg.in(M_val, (size_t)mtot);
    const double *d_dm = dM_val ? sg.in(dM_val, (size_t)mtot) : nullptr;
    double *d_dak = sg.out(dA_k_val, (size_t)ktot);
    double *d_da0 = sg.out(dA_0_val, (size_t)ztot);
    double *d_dmr = dM_resid ? sg.out(dM_resid, (size_t)mtot) : nullptr;
    if (sg.failed) return SAM_ERR_OOM;
    bool ksym = true, zsym = true;  // structurally symmetric sources / targets
    bool one_structure = false;     // every source, every target: one structure each
    {
        std::vector<DevCsr> all(ak);
        all.insert(all.end(), zs.begin(), zs.end());
        std::vector<char> symv, same;
        const std::vector<std::pair<int, int>> ranges{{0, K}, {K, 2 * K}};
        sam_status s = validate_all(h, sc, all, &symv, K > 1 ? &ranges : nullptr, &same);
        if (s != SAM_OK) return s;
        for (size_t q = 0; q < symv.size(); ++q) (q < ak.size() ? ksym : zsym) &= symv[q] != 0;
        one_structure = K > 1 && same[0] && same[1];
    }
    PatternGroup *g = nullptr;
    bool temp = false;
    sam_status s = group_for(h, K, S, &g, &temp);
    if (s != SAM_OK) return s;
    struct GroupGuard {
        PatternGroup *g;
        bool temp;
        ~GroupGuard() {
            if (temp) group_release(g);
        }
    } guard{g, temp};
    // map 0's shadow data serves every map when all structures agree
    const bool shared = one_structure && g->shared;
    const int NS = shared ? n : (int)N;
    int32_t *zcp = nullptr, *zri = nullptr, *zperm = nullptr, *kcp = nullptr, *kri = nullptr, *kperm = nullptr;
    double *zcv = nullptr, *kcv = nullptr;
    int64_t zn = 0, kn = 0;
    if ((s = block_diag_csc(h, sc, zs, n, &zcp, &zri, &zcv, &zperm, &zn, nullptr, zsym)) != SAM_OK) return s;
    if ((s = block_diag_csc(h, sc, ak, n, &kcp, &kri, &kcv, &kperm, &kn, nullptr, ksym)) != SAM_OK) return s;
    int32_t *ish = sc.get<int32_t>((size_t)N * kICap), *icnt = sc.get<int32_t>((size_t)N);
    uint8_t *bin = sc.get<uint8_t>((size_t)N);
    int32_t *colstat = sc.get<int32_t>((size_t)N);
    int64_t *nbcnt = sc.get<int64_t>((size_t)N + 1), *dB_off = sc.get<int64_t>((size_t)N + 1);
    int32_t *work = sc.get<int32_t>((size_t)N);
    int32_t *bin_off = sc.get<int32_t>(kNumBins + 1);
    int64_t *dbase = sc.get<int64_t>((size_t)mtot);
    double *dzval = sc.get<double>((size_t)zn), *dak_csc = sc.get<double>((size_t)kn);
    uint8_t *lrow = sc.get<uint8_t>((size_t)N * kLCap);
    uint8_t *zloc = sc.get<uint8_t>((size_t)N * kZCap);
    if (!ish || !icnt || !bin || !colstat || !nbcnt || !dB_off || !work || !bin_off || !dbase || !dzval ||
        !dak_csc || !lrow || !zloc)
        return SAM_ERR_OOM;
    ShadowTarget tg;
    tg.zcp = zcp;
    tg.zri = zri;
    tg.zbig = 1;
    tg.n = n;
    tg.zloc = zloc;
    if (shadow_and_bins(h, NS, kcp, kri, g->jcp, g->jri, ish, icnt, bin, colstat, nbcnt, lrow, tg) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (shared && (replicate_cols(h, K, n, icnt) != cudaSuccess || replicate_cols(h, K, n, bin) != cudaSuccess ||
                   replicate_cols(h, K, n, colstat) != cudaSuccess || replicate_cols(h, K, n, nbcnt) != cudaSuccess))
        return SAM_ERR_CUDA;
    // map-major order here: the adjoint writes each column's block of dL/dB
    // entries at its own offset, and interleaving the maps scatters those
    // writes (measured 10% slower)
    if (exclusive_scan_i64(h, nbcnt, dB_off, N) != cudaSuccess ||
        build_work_list(h, (int)N, bin, work, bin_off) != cudaSuccess)
        return SAM_ERR_CUDA;
    int64_t nbtot = 0;
    if (cudaMemcpyAsync(&nbtot, dB_off + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SAM_ERR_CUDA;
    double *dB = sc.get<double>((size_t)(nbtot > 0 ? nbtot : 1));
    if (!dB) return SAM_ERR_OOM;
    cudaMemsetAsync(dbase, 0xff, sizeof(int64_t) * (size_t)mtot, st);  // -1: no contribution
    float *kcv32 = nullptr, *zcv32 = nullptr;
    if (precision == SAM_FP32_REFINE) {
        kcv32 = sc.get<float>((size_t)kn);
        zcv32 = sc.get<float>((size_t)zn);
        if (!kcv32 || !zcv32) return SAM_ERR_OOM;
        if (round_to_f32(h, kn, kcv, kcv32) != cudaSuccess || round_to_f32(h, zn, zcv, zcv32) != cudaSuccess)
            return SAM_ERR_CUDA;
    }
    cudaMemsetAsync(dzval, 0, sizeof(double) * (size_t)zn, st);
    if (d_dmr) cudaMemsetAsync(d_dmr, 0, sizeof(double) * (size_t)mtot, st);
    LsqArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n;
    a.kcp = kcp;
    a.kri = kri;
    a.kcv = kcv;
    a.jcp = g->jcp;
    a.jri = g->jri;
    a.ish = ish;
    a.icnt = icnt;
    a.lrow = lrow;
    a.zcp = zcp;
    a.zri = zri;
    a.zcv = zcv;
    a.zbig = 1;
    a.zloc = zloc;
    a.shadow_shared = shared ? 1 : 0;
    a.map_nnz_src = ak[0].nnz;
    a.map_nnz_pat = g->off[1] - g->off[0];
    a.csr_pos = g->csr_pos;
    a.mval = const_cast<double *>(d_m);
    a.kcv32 = kcv32;
    a.zcv32 = zcv32;
    a.colstat = colstat;
    a.work = work;
    a.bin_off = bin_off;
    a.refine_steps = refine_steps;
    a.dmval = d_dm;
    a.resid_weight = resid_weight;
    a.dB = dB;
    a.dB_off = dB_off;
    a.dzval = dzval;
    a.dmres = d_dmr;
    a.dbase = dbase;
    a.znnz = zn;
    if ((s = tape_args(h, sc, g, N, precision, kTapeReplay, a)) != SAM_OK) return s;
    if (launch_adjoint(h, precision, a) != cudaSuccess) return SAM_ERR_CUDA;
    if (adjoint_reduce(h, (int)N, kcp, g->mrp, dbase, dB, dak_csc) != cudaSuccess ||
        permute_scatter_f64(h, kn, kperm, dak_csc, d_dak) != cudaSuccess ||
        permute_scatter_f64(h, zn, zperm, dzval, d_da0) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (status_reduce(h, colstat, N, h->d_flag) != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.has_host_outputs()) return drain_status(h);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

}  // namespace

extern "C" {

sam_status sam_build_backward(sam_handle h, const sam_csr *A_k, const sam_csr *A_0, sam_pattern S, int precision,
                              int refine_steps, const double *M_val, const double *dM_val, double resid_weight,
                              double *dA_k_val, double *dA_0_val, double *dM_resid) {
    if (!S) return SAM_ERR_INVALID_ARG;
    const int64_t off[2] = {0, S->nnz};
    return backward_impl(h, 1, A_k, A_0, &S, precision, refine_steps, off, M_val, dM_val, resid_weight, dA_k_val,
                         dA_0_val, dM_resid);
}

sam_status sam_build_backward_batched(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0,
                                      const sam_pattern *S, int precision, int refine_steps,
                                      const int64_t *M_offsets, const double *M_val, const double *dM_val,
                                      double resid_weight, double *dA_k_val, double *dA_0_val, double *dM_resid) {
    return backward_impl(h, K, A_k, A_0, S, precision, refine_steps, M_offsets, M_val, dM_val, resid_weight,
                         dA_k_val, dA_0_val, dM_resid);
}

sam_status sam_factor_tape_bytes(sam_handle h, int K, const sam_pattern *S, int precision, int64_t *bytes) {
    if (!h || K < 1 || !S || !bytes) return SAM_ERR_INVALID_ARG;
    if (precision != SAM_FP64 && precision != SAM_FP32_REFINE) return SAM_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k)
        if (!S[k] || S[k]->n != S[0]->n) return SAM_ERR_INVALID_ARG;
    if ((int64_t)K * S[0]->n > INT32_MAX - 1) return SAM_ERR_INVALID_ARG;
    PatternGroup *g = nullptr;
    bool temp = false;
    sam_status s = group_for(h, K, S, &g, &temp);
    if (s != SAM_OK) return s;
    {
        Scratch sc(h);
        int64_t *off = nullptr;
        s = tape_layout(h, sc, g, (int64_t)K * S[0]->n, precision, &off, bytes);
    }
    if (temp) group_release(g);
    return s;
}

sam_status sam_set_factor_tape(sam_handle h, int mode, void *buf, int64_t bytes) {
    if (!h) return SAM_ERR_INVALID_ARG;
    if (mode == SAM_TAPE_OFF) {
        h->tape_mode = kTapeOff;
        h->tape_buf = nullptr;
        h->tape_bytes = 0;
        return SAM_OK;
    }
    if ((mode != SAM_TAPE_RECORD && mode != SAM_TAPE_REPLAY) || !buf || bytes < 0 ||
        (reinterpret_cast<uintptr_t>(buf) & 15) != 0)
        return SAM_ERR_INVALID_ARG;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, buf) != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
        (at.type == cudaMemoryTypeDevice && at.device != h->device)) {
        cudaGetLastError();
        return SAM_ERR_INVALID_ARG;
    }
    h->tape_mode = mode == SAM_TAPE_RECORD ? kTapeRecord : kTapeReplay;
    h->tape_buf = buf;
    h->tape_bytes = bytes;
    return SAM_OK;
}

sam_status sam_set_tile_variants(sam_handle h, const int *variants, int count) {
    if (!h || !variants || count != kNumBins) return SAM_ERR_INVALID_ARG;
    for (int b = 0; b < kNumBins; ++b)
        if (variants[b] < 0 || variants[b] >= kTileVariants[b]) return SAM_ERR_INVALID_ARG;
    for (int b = 0; b < kNumBins; ++b) h->variant[b] = variants[b];
    return SAM_OK;
}

sam_status sam_set_bin_schedule(sam_handle h, const int *to, int count) {
    if (!h || !to || count != kNumBins) return SAM_ERR_INVALID_ARG;
    for (int b = 0; b < kNumBins; ++b) {
        const bool ok = b == kBinBig ? to[b] == kBinBig : (to[b] >= b && to[b] < kRegBins);
        if (!ok) return SAM_ERR_INVALID_ARG;
    }
    for (int b = 0; b < kNumBins; ++b) h->sched.to[b] = (uint8_t)to[b];
    return SAM_OK;
}

sam_status sam_get_bin_schedule(sam_handle h, int *to, int count) {
    if (!h || !to || count != kNumBins) return SAM_ERR_INVALID_ARG;
    for (int b = 0; b < kNumBins; ++b) to[b] = h->sched.to[b];
    return SAM_OK;
}

sam_status sam_refine_stats(sam_handle h, int64_t *counts, int count) {
    if (!h || !counts || count != kAutoSteps + 1) return SAM_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(counts, h->d_refine, sizeof(int64_t) * (kAutoSteps + 1), cudaMemcpyDeviceToHost,
                        h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return SAM_ERR_CUDA;
    return SAM_OK;
}

sam_status sam_get_tile_variants(sam_handle h, int *variants, int count) {
    if (!h || !variants || count != kNumBins) return SAM_ERR_INVALID_ARG;
    for (int b = 0; b < kNumBins; ++b) variants[b] = h->variant[b];
    return SAM_OK;
}


sam_status sam_tune(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, const sam_pattern *S, int precision,
                    int refine_steps, const char *cache_path) {
    if (!h || K < 1 || !A_k || !A_0 || !S) return SAM_ERR_INVALID_ARG;
    if (precision != SAM_FP64 && precision != SAM_FP32_REFINE) return SAM_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k)
        if (!S[k]) return SAM_ERR_INVALID_ARG;
    if (precision == SAM_FP64) return SAM_OK;  // one shape per size class: nothing to choose
    std::vector<int64_t> off(K + 1, 0);
    for (int k = 0; k < K; ++k) off[k + 1] = off[k] + S[k]->nnz;
    const int n = A_0->n;
    // outputs of the trial builds: device workspace of this call
    Scratch sc(h);
    int32_t *rp = sc.get<int32_t>((size_t)K * ((size_t)n + 1));
    int32_t *ci = sc.get<int32_t>((size_t)off[K]);
    double *v = sc.get<double>((size_t)off[K]);
    if (!rp || !ci || !v) return SAM_ERR_OOM;
    // the trial builds are timed with the tracing events; keep the caller's
    profile_resolve(h);
    const bool prof = h->profiling;
    const int64_t launches = h->launches;
    double keep_ms[kNumBins];
    int64_t keep_n[kNumBins];
    int saved[kNumBins];
    const BinSchedule saved_sched = h->sched;
    for (int b = 0; b < kNumBins; ++b) {
        keep_ms[b] = h->lsq_ms[b];
        keep_n[b] = h->lsq_n[b];
        saved[b] = h->variant[b];
    }
    BinSchedule ident;
    for (int b = 0; b < kNumBins; ++b) ident.to[b] = (uint8_t)b;
    const int saved_tape = h->tape_mode;  // the trial builds record no factors
    h->tape_mode = kTapeOff;
    auto restore = [&](sam_status result, const int *chosen, const BinSchedule &sched) {
        h->tape_mode = saved_tape;
        h->profiling = prof;
        h->launches = launches;
        h->record_hist = false;
        for (int b = 0; b < kNumBins; ++b) {
            h->lsq_ms[b] = keep_ms[b];
            h->lsq_n[b] = keep_n[b];
            h->variant[b] = result == SAM_OK ? chosen[b] : saved[b];
        }
        h->sched = result == SAM_OK ? sched : saved_sched;
        return result;
    };
    auto build = [&]() {
        return sam_build_batched(h, K, A_k, A_0, S, precision, refine_steps, off.data(), rp, ci, v, nullptr, nullptr,
                                 nullptr);
    };
    // the natural size classes' histogram (identity schedule): the family's key
    int chosen[kNumBins];
    for (int b = 0; b < kNumBins; ++b) chosen[b] = saved[b];
    h->profiling = false;
    h->sched = ident;
    h->record_hist = true;
    sam_status result = build();
    h->record_hist = false;
    if (result == SAM_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) result = SAM_ERR_CUDA;
    if (result != SAM_OK) return restore(result, chosen, saved_sched);
    int64_t hist[kNumBins];
    for (int b = 0; b < kNumBins; ++b) hist[b] = h->h_hist[b + 1] - h->h_hist[b];
    std::string key = tune_key(h, K, n, off[K], precision, refine_steps);
    for (int b = 0; b < kNumBins; ++b) key += " h" + std::to_string((long long)hist[b]);
    BinSchedule sched = ident;
    {
        int to[kNumBins];
        if (tune_lookup(cache_path, key, chosen, to)) {
            for (int b = 0; b < kNumBins; ++b) sched.to[b] = (uint8_t)to[b];
            return restore(SAM_OK, chosen, sched);
        }
    }
    constexpr int kTrials = 3;
    // mean time per build of every size class's launches under the current
    // variants and schedule (one warm-up, kTrials timed builds)
    double cls_ms[kNumBins];
    auto trial = [&]() -> sam_status {
        h->profiling = false;
        sam_status r = build();
        if (r != SAM_OK) return r;
        for (int b = 0; b < kNumBins; ++b) {
            h->lsq_ms[b] = 0.0;
            h->lsq_n[b] = 0;
        }
        h->profiling = true;
        for (int t = 0; t < kTrials && r == SAM_OK; ++t) r = build();
        if (r == SAM_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) r = SAM_ERR_CUDA;
        profile_resolve(h);
        h->profiling = false;
        for (int b = 0; b < kNumBins; ++b) cls_ms[b] = h->lsq_ms[b] / kTrials;
        return r;
    };
    // 1. tile shapes: every size class tries its variant `var` (the last one
    //    if it has fewer); the fastest launch per class wins
    double best[kNumBins];
    for (int b = 0; b < kNumBins; ++b) {
        best[b] = 1e300;
        chosen[b] = 0;
    }
    int max_var = 1;
    for (int b = 0; b < kNumBins; ++b) max_var = std::max(max_var, kTileVariants[b]);
    for (int var = 0; var < max_var && result == SAM_OK; ++var) {
        for (int b = 0; b < kNumBins; ++b) h->variant[b] = std::min(var, kTileVariants[b] - 1);
        result = trial();
        for (int b = 0; b < kNumBins && result == SAM_OK; ++b) {
            if (h->variant[b] != var || hist[b] == 0) continue;
            if (cls_ms[b] < best[b]) {
                best[b] = cls_ms[b];
                chosen[b] = var;
            }
        }
    }
    // 2. bin schedule: fold each small register class into the next one that
    //    still solves columns (fewer launches, fuller waves), greedily from
    //    the smallest, kept when the summed launch time drops by 1% or more
    if (result == SAM_OK) {
        for (int b = 0; b < kNumBins; ++b) h->variant[b] = chosen[b];
        result = trial();
        double cur = 0.0;
        for (int b = 0; b < kNumBins; ++b) cur += cls_ms[b];
        for (int b = 0; b + 1 < kRegBins && result == SAM_OK; ++b) {
            if (hist[b] == 0 || sched.to[b] != b) continue;
            BinSchedule cand = sched;
            const uint8_t next = cand.to[b + 1];
            for (int c = 0; c < kRegBins; ++c)
                if (cand.to[c] == b) cand.to[c] = next;
            h->sched = cand;
            result = trial();
            double tot = 0.0;
            for (int c = 0; c < kNumBins; ++c) tot += cls_ms[c];
            if (result == SAM_OK && tot <= 0.99 * cur) {
                sched = cand;
                cur = tot;
            }
            h->sched = sched;
        }
    }
    if (result != SAM_OK) return restore(result, chosen, saved_sched);
    restore(SAM_OK, chosen, sched);
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (!f) return SAM_ERR_INVALID_ARG;
        fprintf(f, "%s", key.c_str());
        for (int b = 0; b < kNumBins; ++b) fprintf(f, " %d", chosen[b]);
        for (int b = 0; b < kNumBins; ++b) fprintf(f, " %d", (int)sched.to[b]);
        fprintf(f, "\n");
        fclose(f);
    }
    return SAM_OK;
}

sam_status sam_profile(sam_handle h, int enable) {
    if (!h) return SAM_ERR_INVALID_ARG;
    profile_resolve(h);
    h->profiling = enable != 0;
    h->launches = 0;
    for (int b = 0; b < kNumBins; ++b) {
        h->lsq_ms[b] = 0.0;
        h->lsq_n[b] = 0;
    }
    return SAM_OK;
}

sam_status sam_profile_read(sam_handle h, int64_t *launches, double *lsq_ms, int64_t *lsq_launches) {
    if (!h) return SAM_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
    profile_resolve(h);
    if (launches) *launches = h->launches;
    for (int b = 0; b < kNumBins; ++b) {
        if (lsq_ms) lsq_ms[b] = h->lsq_ms[b];
        if (lsq_launches) lsq_launches[b] = h->lsq_n[b];
    }
    return SAM_OK;
}

sam_status sam_peak_flops(sam_handle h, double ms, double *fp32_flops, double *fp64_flops) {
    if (!h || ms <= 0) return SAM_ERR_INVALID_ARG;
    if (peak_fma(h, ms, fp32_flops, fp64_flops) != cudaSuccess) return SAM_ERR_CUDA;
    return drain_status(h);
}

}  // extern "C"

namespace {

void plan_free(sam_plan p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (void *q : p->mem) pool_free(p->h, q);
    if (p->g) group_release(p->g);
    delete p;
}

}  // namespace

extern "C" {

sam_status sam_plan_create(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, int n_targets,
                           const sam_pattern *S, int precision, int refine_steps, const int64_t *M_offsets,
                           int32_t *M_row_ptr, int32_t *M_col_idx, double *M_val, int32_t *col_status, double *res2,
                           double *fro2, sam_plan *out) {
    if (!out) return SAM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h || K < 1 || !A_k || !A_0 || !S || !M_offsets || !M_row_ptr || !M_col_idx || !M_val)
        return SAM_ERR_INVALID_ARG;
    if (n_targets != 1 && n_targets != K) return SAM_ERR_INVALID_ARG;
    if (precision != SAM_FP64 && precision != SAM_FP32_REFINE) return SAM_ERR_INVALID_ARG;
    if (refine_steps < SAM_REFINE_AUTO || refine_steps > 4) return SAM_ERR_INVALID_ARG;
    const int NT = n_targets;
    const int n = A_0[0].n;
    int64_t ktot = 0, ztot = 0;
    auto dev_csr = [](const sam_csr &a) {
        return is_device_ptr(a.row_ptr) && (a.nnz == 0 || (is_device_ptr(a.col_idx) && is_device_ptr(a.val)));
    };
    for (int t = 0; t < NT; ++t) {
        if (check_csr_arg(&A_0[t], true) != SAM_OK || A_0[t].n != n || !dev_csr(A_0[t])) return SAM_ERR_INVALID_ARG;
        ztot += A_0[t].nnz;
    }
    if (M_offsets[0] != 0) return SAM_ERR_INVALID_ARG;
    for (int k = 0; k < K; ++k) {
        if (check_csr_arg(&A_k[k], true) != SAM_OK || A_k[k].n != n || !S[k] || S[k]->n != n || !dev_csr(A_k[k]))
            return SAM_ERR_INVALID_ARG;
        if (M_offsets[k + 1] - M_offsets[k] != S[k]->nnz) return SAM_ERR_INVALID_ARG;
        ktot += A_k[k].nnz;
    }
    const int64_t N = (int64_t)K * n;
    const int64_t total_nnz = M_offsets[K];
    if (N > INT32_MAX - 1 || ktot > INT32_MAX || ztot > INT32_MAX || total_nnz > INT32_MAX)
        return SAM_ERR_INVALID_ARG;
    if (!is_device_ptr(M_row_ptr) || (total_nnz > 0 && (!is_device_ptr(M_col_idx) || !is_device_ptr(M_val))) ||
        (col_status && !is_device_ptr(col_status)) || (res2 && !is_device_ptr(res2)) || (fro2 && !is_device_ptr(fro2)))
        return SAM_ERR_INVALID_ARG;
    sam_plan p = new (std::nothrow) sam_plan_t;
    if (!p) return SAM_ERR_OOM;
    p->h = h;
    struct Guard {
        sam_plan p;
        ~Guard() { plan_free(p); }
    } guard{p};
    cudaStream_t st = h->stream;
    Scratch keep(h), tmp(h);
    std::vector<DevCsr> zs(NT), ak(K);
    for (int t = 0; t < NT; ++t) zs[t] = DevCsr{A_0[t].n, A_0[t].nnz, A_0[t].row_ptr, A_0[t].col_idx, A_0[t].val};
    for (int k = 0; k < K; ++k) ak[k] = DevCsr{A_k[k].n, A_k[k].nnz, A_k[k].row_ptr, A_k[k].col_idx, A_k[k].val};
    bool ksym = true, zsym = true;  // structurally symmetric sources / targets
    bool one_structure = false;     // every source, every target: one structure each
    {
        std::vector<DevCsr> all(ak);
        all.insert(all.end(), zs.begin(), zs.end());
        std::vector<char> symv, same;
        const std::vector<std::pair<int, int>> ranges{{0, K}, {K, K + NT}};
        sam_status s = validate_all(h, tmp, all, &symv, K > 1 ? &ranges : nullptr, &same);
        if (s != SAM_OK) return s;
        for (size_t q = 0; q < symv.size(); ++q) (q < ak.size() ? ksym : zsym) &= symv[q] != 0;
        one_structure = K > 1 && same[0] && same[1];
    }
    {
        bool temp = false;
        sam_status s = group_for(h, K, S, &p->g, &temp);
        if (s != SAM_OK) {
            p->g = nullptr;
            return s;
        }
        if (!temp) p->g->refs++;
    }
    PatternGroup *g = p->g;
    // the same sharing of structure work, and the same work order, as the
    // direct call (so replays equal it bit for bit)
    const bool shared = one_structure && g->shared;
    const int NS = shared ? n : (int)N;
    // ---- value-independent work, done once
    int32_t *zcp = nullptr, *zri = nullptr, *zperm = nullptr, *kcp = nullptr, *kri = nullptr, *kperm = nullptr;
    double *zcv = nullptr, *kcv = nullptr;
    int64_t zn = 0, kn = 0;
    sam_status s = block_diag_csc(h, keep, zs, n, &zcp, &zri, &zcv, &zperm, &zn, &tmp, zsym);
    if (s != SAM_OK) return s;
    if ((s = block_diag_csc(h, keep, ak, n, &kcp, &kri, &kcv, &kperm, &kn, &tmp, ksym)) != SAM_OK) return s;
    int32_t *ish = keep.get<int32_t>((size_t)N * kICap), *icnt = keep.get<int32_t>((size_t)N);
    // (automatic refinement reads the size classes at every replay)
    uint8_t *bin = refine_steps < 0 && precision == SAM_FP32_REFINE ? keep.get<uint8_t>((size_t)N)
                                                                     : tmp.get<uint8_t>((size_t)N);
    int32_t *work = keep.get<int32_t>((size_t)N);
    int32_t *bin_off = keep.get<int32_t>(kNumBins + 1);
    int32_t *d_st = col_status ? col_status : keep.get<int32_t>((size_t)N);
    double *d_r2 = res2 ? res2 : keep.get<double>((size_t)N);
    uint8_t *lrow = keep.get<uint8_t>((size_t)N * kLCap);
    uint8_t *zloc = keep.get<uint8_t>((size_t)N * kZCap);
    if (!zloc) return SAM_ERR_OOM;
    float *kcv32 = nullptr, *zcv32 = nullptr;
    if (precision == SAM_FP32_REFINE) {
        kcv32 = keep.get<float>((size_t)kn);
        zcv32 = keep.get<float>((size_t)zn);
    }
    double *seg_work = fro2 ? keep.get<double>(segmented_sum_workspace(K)) : nullptr;
    // automatic refinement or a fixed number of steps >= 1: the FP64
    // re-solve of the columns that miss the accuracy target is captured too
    const bool autoref = precision == SAM_FP32_REFINE && refine_steps != 0;
    uint8_t *refine_used = autoref ? keep.get<uint8_t>((size_t)N) : nullptr;
    int32_t *work2 = autoref ? keep.get<int32_t>((size_t)N) : nullptr;
    int32_t *bin_off2 = autoref ? keep.get<int32_t>(kNumBins + 1) : nullptr;
    if (autoref && (!refine_used || !work2 || !bin_off2)) return SAM_ERR_OOM;
    // automatic refinement: the two-step launch's own lists (the first
    // launch's work list is read again at every replay)
    RedoLists redo;
    if (refine_steps < 0 && precision == SAM_FP32_REFINE) {
        redo.bin = bin;
        redo.bins2 = keep.get<uint8_t>((size_t)N);
        redo.work = keep.get<int32_t>((size_t)N);
        redo.bin_off = keep.get<int32_t>(kNumBins + 1);
        redo.ws = keep.get<int32_t>(2 * kNumBins);
        if (!redo.bins2 || !redo.work || !redo.bin_off || !redo.ws) return SAM_ERR_OOM;
    }
    // value sources: per-matrix pointers and CSC offsets
    std::vector<const double *> kptr(K), zptr(NT);
    std::vector<int64_t> koff(K + 1, 0), zoff(NT + 1, 0);
    for (int k = 0; k < K; ++k) {
        kptr[k] = A_k[k].val;
        koff[k + 1] = koff[k] + A_k[k].nnz;
    }
    for (int t = 0; t < NT; ++t) {
        zptr[t] = A_0[t].val;
        zoff[t + 1] = zoff[t] + A_0[t].nnz;
    }
    const double **d_kptr = keep.get<const double *>(K), **d_zptr = keep.get<const double *>(NT);
    int64_t *d_koff = keep.get<int64_t>(K + 1), *d_zoff = keep.get<int64_t>(NT + 1);
    if (!ish || !icnt || !bin || !work || !bin_off || !d_st || !d_r2 || !lrow ||
        (precision == SAM_FP32_REFINE && (!kcv32 || !zcv32)) || (fro2 && !seg_work) || !d_kptr || !d_zptr ||
        !d_koff || !d_zoff)
        return SAM_ERR_OOM;
    cudaMemcpyAsync(d_kptr, kptr.data(), sizeof(double *) * K, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_zptr, zptr.data(), sizeof(double *) * NT, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_koff, koff.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_zoff, zoff.data(), sizeof(int64_t) * (NT + 1), cudaMemcpyHostToDevice, st);
    ShadowTarget tg;
    tg.zcp = zcp;
    tg.zri = zri;
    tg.zbig = NT > 1 ? 1 : 0;
    tg.n = n;
    tg.zloc = zloc;
    if (shadow_and_bins(h, NS, kcp, kri, g->jcp, g->jri, ish, icnt, bin, d_st, nullptr, lrow, tg) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (shared && (replicate_cols(h, K, n, icnt) != cudaSuccess || replicate_cols(h, K, n, bin) != cudaSuccess ||
                   replicate_cols(h, K, n, d_st) != cudaSuccess))
        return SAM_ERR_CUDA;
    if ((shared ? interleaved_work_list(h, tmp, K, n, bin, work, bin_off)
                : build_work_list(h, (int)N, bin, work, bin_off)) != cudaSuccess ||
        split_map_structure(h, K, n, g->mrp, g->mci, M_row_ptr, M_col_idx) != cudaSuccess)
        return SAM_ERR_CUDA;
    // shadow failures (rank / unsupported) are structural: report them now
    if (status_reduce(h, d_st, N, h->d_flag) != cudaSuccess) return SAM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SAM_ERR_CUDA;
    // ---- value-dependent steps, captured once on a private stream
    LsqArgs a;
    memset(&a, 0, sizeof(a));
    a.kcv32 = kcv32;
    a.zcv32 = zcv32;
    a.n = n;
    a.kcp = kcp;
    a.kri = kri;
    a.kcv = kcv;
    a.jcp = g->jcp;
    a.jri = g->jri;
    a.ish = ish;
    a.icnt = icnt;
    a.lrow = lrow;
    a.zcp = zcp;
    a.zri = zri;
    a.zcv = zcv;
    a.zbig = NT > 1 ? 1 : 0;
    a.zloc = zloc;
    a.shadow_shared = shared ? 1 : 0;
    a.map_nnz_src = ak[0].nnz;
    a.map_nnz_pat = g->off[1] - g->off[0];
    a.csr_pos = g->csr_pos;
    a.mval = M_val;
    a.colres = d_r2;
    a.colstat = d_st;
    a.work = work;
    a.bin_off = bin_off;
    a.refine_steps = refine_steps;
    a.refine_used = refine_used;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return SAM_ERR_CUDA;
    const bool prof = h->profiling;
    const int64_t launches0 = h->launches;
    h->profiling = false;
    h->stream = cs;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // the shadow status of each column is kept in d_st; the solve overwrites it per column
        bool ok = gather_values(h, kn, K, d_koff, d_kptr, kperm, kcv, kcv32) == cudaSuccess &&
                  gather_values(h, zn, NT, d_zoff, d_zptr, zperm, zcv, zcv32) == cudaSuccess &&
                  cudaMemsetAsync(M_val, 0, sizeof(double) * (size_t)total_nnz, cs) == cudaSuccess &&
                  cudaMemsetAsync(d_r2, 0, sizeof(double) * (size_t)N, cs) == cudaSuccess &&
                  (!autoref || cudaMemsetAsync(refine_used, 0, (size_t)N, cs) == cudaSuccess) &&
                  launch_lsq(h, precision, a) == cudaSuccess &&
                  (!autoref || launch_refine_fallback(h, a, (int)N, work2, bin_off2, h->d_refine, redo) == cudaSuccess) &&
                  status_reduce(h, d_st, N, h->d_flag) == cudaSuccess &&
                  (!fro2 || segmented_sum_f64(h, d_r2, K, n, fro2, false, seg_work) == cudaSuccess);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        p->graph = graph;
        if (!ok && e == cudaSuccess) e = cudaErrorUnknown;
    }
    h->stream = st;
    h->profiling = prof;
    p->launches = h->launches - launches0;
    h->launches = launches0;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || !p->graph) {
        cudaGetLastError();
        return SAM_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return SAM_ERR_CUDA;
    }
    p->mem = keep.release();
    *out = p;
    guard.p = nullptr;
    return drain_status(h);
}

sam_status sam_plan_execute(sam_plan p) {
    if (!p || !p->exec) return SAM_ERR_INVALID_ARG;
    if (cudaGraphLaunch(p->exec, p->h->stream) != cudaSuccess) {
        cudaGetLastError();
        return SAM_ERR_CUDA;
    }
    p->h->launches += p->launches;
    return SAM_OK;
}

sam_status sam_plan_launches(sam_plan p, int64_t *launches) {
    if (!p || !launches) return SAM_ERR_INVALID_ARG;
    *launches = p->launches;
    return SAM_OK;
}

sam_status sam_plan_destroy(sam_plan p) {
    if (!p) return SAM_ERR_INVALID_ARG;
    cudaStreamSynchronize(p->h->stream);
    plan_free(p);
    return SAM_OK;
}

}  // extern "C"

