// api.cu -- the C ABI of libsam (declared in include/sam.h): handles, the
// stream-ordered device workspace, host/device argument staging, and the
// orchestration of the pattern, build, residual and apply pipelines.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

struct sam_handle_t {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sms = 1;
    uint32_t flags = 0;
    cudaMemPool_t pool = nullptr;
    int32_t *d_flag = nullptr;   // sticky device status word
    int32_t *h_flag = nullptr;   // pinned mirror
    sam_status host_sticky = SAM_OK;
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
};

struct sam_pattern_t {
    sam_handle h = nullptr;
    int n = 0;
    int64_t nnz = 0;
    int32_t *jcp = nullptr, *jri = nullptr;      // pattern, CSC (= CSC structure of the map)
    int32_t *mrp = nullptr, *mci = nullptr;      // CSR structure of the map
    int32_t *csr_pos = nullptr;                  // CSC entry -> CSR position
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
    };
    std::vector<Out> outs;
    bool failed = false;
    Stager(Scratch &s, cudaStream_t stream) : sc(s), st(stream) {}
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
        outs.push_back({(void *)p, (const void *)d, sizeof(T) * count});
        return d;
    }
    bool has_host_outputs() const { return !outs.empty(); }
    cudaError_t finish() {
        for (auto &o : outs) {
            cudaError_t e = cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

struct DevCsr {
    int n = 0;
    int64_t nnz = 0;
    const int32_t *rp = nullptr, *ci = nullptr;
    const double *v = nullptr;
};

sam_status check_csr_arg(const sam_csr *A, bool need_val) {
    if (!A || A->n < 0 || A->nnz < 0 || A->nnz > INT32_MAX || !A->row_ptr || (A->nnz > 0 && !A->col_idx) ||
        (need_val && A->nnz > 0 && !A->val))
        return SAM_ERR_INVALID_ARG;
    return SAM_OK;
}

DevCsr stage_csr(Stager &sg, const sam_csr *A, bool with_val) {
    DevCsr d;
    d.n = A->n;
    d.nnz = A->nnz;
    d.rp = sg.in(A->row_ptr, (size_t)A->n + 1);
    d.ci = sg.in(A->col_idx, (size_t)A->nnz);
    d.v = with_val ? sg.in(A->val, (size_t)A->nnz) : nullptr;
    return d;
}

// Reads and clears the sticky device status (synchronises the stream).
sam_status drain_status(sam_handle h) {
    if (cudaMemcpyAsync(h->h_flag, h->d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
    sam_status s = *h->h_flag;
    if (s != SAM_OK) cudaMemsetAsync(h->d_flag, 0, sizeof(int32_t), h->stream);
    if (s == SAM_OK && h->host_sticky != SAM_OK) s = h->host_sticky;
    h->host_sticky = SAM_OK;
    return s;
}

// Validates CSR structures on the device; synchronises once.
sam_status validate_all(sam_handle h, const std::vector<DevCsr> &ms) {
    if (h->flags & SAM_FLAG_TRUSTED) return SAM_OK;
    int32_t *flag = (int32_t *)pool_alloc(h, sizeof(int32_t));
    if (!flag) return SAM_ERR_OOM;
    cudaMemsetAsync(flag, 0, sizeof(int32_t), h->stream);
    for (auto &m : ms)
        if (validate_csr(h, m.n, m.nnz, m.rp, m.ci, flag) != cudaSuccess) return SAM_ERR_CUDA;
    int32_t hv = 0;
    cudaMemcpyAsync(h->h_flag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    pool_free(h, flag);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
    hv = *h->h_flag;
    return hv ? (sam_status)hv : SAM_OK;
}

__global__ void scatter_inverse_kernel(int64_t nnz, const int32_t *perm, int32_t *pos) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) pos[perm[p]] = (int32_t)p;
}

// Pattern object from a CSC pattern already on the device (takes ownership
// of jcp / jri, which must come from the handle's pool).
sam_status finish_pattern(sam_handle h, int n, int64_t nnz, int32_t *jcp, int32_t *jri, sam_pattern *out) {
    sam_pattern S = new (std::nothrow) sam_pattern_t;
    if (!S) return SAM_ERR_OOM;
    S->h = h;
    S->n = n;
    S->nnz = nnz;
    S->jcp = jcp;
    S->jri = jri;
    S->mrp = (int32_t *)pool_alloc(h, sizeof(int32_t) * ((size_t)n + 1));
    S->mci = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    S->csr_pos = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    int32_t *perm = (int32_t *)pool_alloc(h, sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    if (!S->mrp || !S->mci || !S->csr_pos || !perm) {
        pool_free(h, perm);
        sam_pattern_destroy(S);
        return SAM_ERR_OOM;
    }
    // the CSC of the map read as the CSR of its transpose; transposing it
    // gives the CSR of the map, and perm[p] = CSC entry of CSR position p
    if (csr_to_csc(h, n, nnz, jcp, jri, nullptr, S->mrp, S->mci, nullptr, perm) != cudaSuccess) {
        pool_free(h, perm);
        sam_pattern_destroy(S);
        return SAM_ERR_CUDA;
    }
    if (nnz > 0) {
        scatter_inverse_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, h->stream>>>(nnz, perm, S->csr_pos);
        count_launch(h);
    }
    pool_free(h, perm);
    if (cudaGetLastError() != cudaSuccess) {
        sam_pattern_destroy(S);
        return SAM_ERR_CUDA;
    }
    *out = S;
    return SAM_OK;
}

__global__ void validate_pattern_kernel(int n, int64_t nnz, const int32_t *cp, const int32_t *ri, int32_t *flag) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0 && (cp[0] != 0 || (int64_t)cp[n] != nnz)) atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
    if (j >= n) return;
    int b = cp[j], e = cp[j + 1];
    if (e <= b || b < 0 || (int64_t)e > nnz) {  // every column must be nonempty
        atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
        return;
    }
    for (int t = b; t < e; ++t)
        if (ri[t] < 0 || ri[t] >= n || (t > b && ri[t] <= ri[t - 1])) {
            atomicCAS(flag, 0, SAM_ERR_BAD_CSR);
            return;
        }
}

__global__ void rowptr_rebase_kernel(int n, const int32_t *src, int32_t *dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) dst[i] = src[i];
}

}  // namespace

extern "C" {

void sam_limits(int32_t *max_rows, int32_t *max_cols) {
    if (max_rows) *max_rows = kICap;
    if (max_cols) *max_cols = kJCap;
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
        cudaMallocHost(&h->h_flag, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        if (h->d_flag) cudaFree(h->d_flag);
        cudaMemPoolDestroy(h->pool);
        delete h;
        return SAM_ERR_OOM;
    }
    cudaMemset(h->d_flag, 0, sizeof(int32_t));
    *h->h_flag = 0;
    *out = h;
    return SAM_OK;
}

sam_status sam_destroy(sam_handle h) {
    if (!h) return SAM_ERR_INVALID_ARG;
    cudaStreamSynchronize(h->stream);
    h->profiling = false;
    profile_resolve(h);
    cudaFree(h->d_flag);
    cudaFreeHost(h->h_flag);
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
    for (int k = 0; k < K; ++k) {
        out[k] = nullptr;
        if (check_csr_arg(&A[k], false) != SAM_OK || A[k].n != A[0].n) return SAM_ERR_INVALID_ARG;
    }
    const int n = A[0].n;
    Scratch sc(h);
    Stager sg(sc, h->stream);
    std::vector<DevCsr> d(K);
    for (int k = 0; k < K; ++k) d[k] = stage_csr(sg, &A[k], false);
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, d);
    if (s != SAM_OK) return s;
    std::vector<int32_t *> kcp(K), kri(K);
    for (int k = 0; k < K; ++k) {
        kcp[k] = sc.get<int32_t>((size_t)n + 1);
        kri[k] = sc.get<int32_t>((size_t)d[k].nnz);
        if (!kcp[k] || !kri[k]) return SAM_ERR_OOM;
        if (csr_to_csc(h, n, d[k].nnz, d[k].rp, d[k].ci, nullptr, kcp[k], kri[k], nullptr, nullptr) != cudaSuccess)
            return SAM_ERR_CUDA;
    }
    std::vector<int32_t *> jcp(K), jri(K);
    std::vector<int64_t> nnz(K);
    s = level_pattern_batched(h, K, n, kcp.data(), kri.data(), level, jcp.data(), jri.data(), nnz.data());
    if (s != SAM_OK) return s;
    for (int k = 0; k < K; ++k) {
        s = finish_pattern(h, n, nnz[k], jcp[k], jri[k], &out[k]);
        if (s != SAM_OK) {
            for (int q = 0; q < k; ++q) {
                sam_pattern_destroy(out[q]);
                out[q] = nullptr;
            }
            return s;
        }
    }
    return drain_status(h);
}

sam_status sam_pattern_build(sam_handle h, const sam_csr *A_k, int level, sam_pattern *out) {
    return sam_pattern_build_batched(h, 1, A_k, level, out);
}

sam_status sam_pattern_from_csc(sam_handle h, int32_t n, int64_t nnz, const int32_t *colptr, const int32_t *rowidx,
                                sam_pattern *out) {
    if (!h || !out || n < 0 || nnz < n || nnz > INT32_MAX || !colptr || !rowidx) return SAM_ERR_INVALID_ARG;
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
    int32_t *flag = (int32_t *)pool_alloc(h, sizeof(int32_t));
    cudaMemsetAsync(flag, 0, sizeof(int32_t), h->stream);
    validate_pattern_kernel<<<(n + 255) / 256 > 0 ? (n + 255) / 256 : 1, 256, 0, h->stream>>>(n, nnz, jcp, jri, flag);
    count_launch(h);
    cudaMemcpyAsync(h->h_flag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    pool_free(h, flag);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SAM_ERR_CUDA;
    if (*h->h_flag != 0) {
        sam_status s = *h->h_flag;
        *h->h_flag = 0;
        pool_free(h, jcp);
        pool_free(h, jri);
        return s;
    }
    return finish_pattern(h, n, nnz, jcp, jri, out);
}

sam_status sam_pattern_get(sam_pattern S, int32_t *n, int64_t *nnz, const int32_t **colptr, const int32_t **rowidx) {
    if (!S) return SAM_ERR_INVALID_ARG;
    if (n) *n = S->n;
    if (nnz) *nnz = S->nnz;
    if (colptr) *colptr = S->jcp;
    if (rowidx) *rowidx = S->jri;
    return SAM_OK;
}

sam_status sam_pattern_destroy(sam_pattern S) {
    if (!S) return SAM_ERR_INVALID_ARG;
    sam_handle h = S->h;
    pool_free(h, S->jcp);
    pool_free(h, S->jri);
    pool_free(h, S->mrp);
    pool_free(h, S->mci);
    pool_free(h, S->csr_pos);
    delete S;
    return SAM_OK;
}

sam_status sam_build_batched(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, const sam_pattern *S,
                             int precision, int refine_steps, const int64_t *M_offsets, int32_t *M_row_ptr,
                             int32_t *M_col_idx, double *M_val, int32_t *col_status, double *res2, double *fro) {
    if (!h || K < 1 || !A_k || !A_0 || !S || !M_offsets || !M_row_ptr || !M_col_idx || !M_val)
        return SAM_ERR_INVALID_ARG;
    if (precision != SAM_FP64 && precision != SAM_FP32_REFINE) return SAM_ERR_INVALID_ARG;
    if (refine_steps < 0 || refine_steps > 4) return SAM_ERR_INVALID_ARG;
    if (check_csr_arg(A_0, true) != SAM_OK) return SAM_ERR_INVALID_ARG;
    const int n = A_0->n;
    for (int k = 0; k < K; ++k) {
        if (check_csr_arg(&A_k[k], true) != SAM_OK || A_k[k].n != n || !S[k] || S[k]->n != n)
            return SAM_ERR_INVALID_ARG;
        if (M_offsets[k + 1] - M_offsets[k] != S[k]->nnz || M_offsets[k] < 0) return SAM_ERR_INVALID_ARG;
    }
    const int64_t total_nnz = M_offsets[K];
    cudaStream_t st = h->stream;
    Scratch sc(h);
    Stager sg(sc, st);
    DevCsr z = stage_csr(sg, A_0, true);
    std::vector<DevCsr> ak(K);
    for (int k = 0; k < K; ++k) ak[k] = stage_csr(sg, &A_k[k], true);
    int32_t *d_rp = sg.out(M_row_ptr, (size_t)K * ((size_t)n + 1));
    int32_t *d_ci = sg.out(M_col_idx, (size_t)total_nnz);
    double *d_v = sg.out(M_val, (size_t)total_nnz);
    int32_t *d_st = col_status ? sg.out(col_status, (size_t)K * (size_t)n) : nullptr;
    double *d_r2 = res2 ? sg.out(res2, (size_t)K * (size_t)n) : nullptr;
    if (sg.failed) return SAM_ERR_OOM;
    {
        std::vector<DevCsr> all(ak);
        all.push_back(z);
        sam_status s = validate_all(h, all);
        if (s != SAM_OK) return s;
    }
    // CSC of the target (shared) and of every source
    int32_t *zcp = sc.get<int32_t>((size_t)n + 1), *zri = sc.get<int32_t>((size_t)z.nnz);
    double *zcv = sc.get<double>((size_t)z.nnz);
    if (!zcp || !zri || !zcv) return SAM_ERR_OOM;
    if (csr_to_csc(h, n, z.nnz, z.rp, z.ci, z.v, zcp, zri, zcv, nullptr) != cudaSuccess) return SAM_ERR_CUDA;
    if (!d_st) d_st = sc.get<int32_t>((size_t)K * n);
    if (!d_r2) d_r2 = sc.get<double>((size_t)K * n);
    if (!d_st || !d_r2) return SAM_ERR_OOM;
    std::vector<MapDev> maps(K);
    std::vector<const uint8_t *> bins(K);
    for (int k = 0; k < K; ++k) {
        int32_t *kcp = sc.get<int32_t>((size_t)n + 1), *kri = sc.get<int32_t>((size_t)ak[k].nnz);
        double *kcv = sc.get<double>((size_t)ak[k].nnz);
        int32_t *ish = sc.get<int32_t>((size_t)n * kICap), *icnt = sc.get<int32_t>((size_t)n);
        uint8_t *bin = sc.get<uint8_t>((size_t)n);
        if (!kcp || !kri || !kcv || !ish || !icnt || !bin) return SAM_ERR_OOM;
        if (csr_to_csc(h, n, ak[k].nnz, ak[k].rp, ak[k].ci, ak[k].v, kcp, kri, kcv, nullptr) != cudaSuccess)
            return SAM_ERR_CUDA;
        int32_t *colstat = d_st + (size_t)k * n;
        if (shadow_and_bins(h, n, kcp, kri, S[k]->jcp, S[k]->jri, precision, ish, icnt, bin, colstat) != cudaSuccess)
            return SAM_ERR_CUDA;
        MapDev &m = maps[k];
        memset(&m, 0, sizeof(m));
        m.kcp = kcp;
        m.kri = kri;
        m.kcv = kcv;
        m.jcp = S[k]->jcp;
        m.jri = S[k]->jri;
        m.ish = ish;
        m.icnt = icnt;
        m.csr_pos = S[k]->csr_pos;
        m.mval = d_v + M_offsets[k];
        m.colres = d_r2 + (size_t)k * n;
        m.colstat = colstat;
        bins[k] = bin;
    }
    int2 *work = sc.get<int2>((size_t)K * n);
    int32_t *bin_off = sc.get<int32_t>(kNumBins + 1);
    int32_t *tickets = sc.get<int32_t>(kNumBins);
    MapDev *maps_dev = sc.get<MapDev>((size_t)K);
    if (!work || !bin_off || !tickets || !maps_dev) return SAM_ERR_OOM;
    if (cudaMemcpyAsync(maps_dev, maps.data(), sizeof(MapDev) * K, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SAM_ERR_CUDA;
    if (build_work_lists(h, K, n, bins.data(), work, bin_off) != cudaSuccess) return SAM_ERR_CUDA;
    cudaMemsetAsync(d_v, 0, sizeof(double) * (size_t)total_nnz, st);
    cudaMemsetAsync(d_r2, 0, sizeof(double) * (size_t)K * n, st);
    if (launch_lsq(h, precision, refine_steps, 0, maps_dev, zcp, zri, zcv, work, bin_off, tickets) != cudaSuccess)
        return SAM_ERR_CUDA;
    // CSR structure of every map
    for (int k = 0; k < K; ++k) {
        cudaMemcpyAsync(d_rp + (size_t)k * (n + 1), S[k]->mrp, sizeof(int32_t) * ((size_t)n + 1),
                        cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(d_ci + M_offsets[k], S[k]->mci, sizeof(int32_t) * (size_t)S[k]->nnz, cudaMemcpyDeviceToDevice,
                        st);
    }
    if (status_reduce(h, d_st, (int64_t)K * n, h->d_flag) != cudaSuccess) return SAM_ERR_CUDA;
    double *fro_dev = nullptr;
    if (fro) {
        fro_dev = sc.get<double>((size_t)K);
        if (!fro_dev) return SAM_ERR_OOM;
        for (int k = 0; k < K; ++k)
            if (sum_f64(h, d_r2 + (size_t)k * n, n, fro_dev + k, false) != cudaSuccess) return SAM_ERR_CUDA;
    }
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    if (fro) {
        std::vector<double> f2(K);
        if (cudaMemcpyAsync(f2.data(), fro_dev, sizeof(double) * K, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SAM_ERR_CUDA;
        sam_status s = drain_status(h);
        for (int k = 0; k < K; ++k) fro[k] = sqrt(f2[k]);
        return s;
    }
    if (sg.has_host_outputs()) return drain_status(h);
    return cudaGetLastError() == cudaSuccess ? SAM_OK : SAM_ERR_CUDA;
}

sam_status sam_build(sam_handle h, const sam_csr *A_k, const sam_csr *A_0, sam_pattern S, int precision,
                     int refine_steps, int32_t *M_row_ptr, int32_t *M_col_idx, double *M_val, int32_t *col_status,
                     double *res2) {
    if (!S) return SAM_ERR_INVALID_ARG;
    int64_t off[2] = {0, S->nnz};
    return sam_build_batched(h, 1, A_k, A_0, &S, precision, refine_steps, off, M_row_ptr, M_col_idx, M_val,
                             col_status, res2, nullptr);
}

sam_status sam_residual(sam_handle h, const sam_csr *A_k, const sam_csr *M_k, const sam_csr *A_0, double *fro,
                        double *rel) {
    if (!h || check_csr_arg(A_k, true) || check_csr_arg(M_k, true) || check_csr_arg(A_0, true)) return SAM_ERR_INVALID_ARG;
    const int n = A_k->n;
    if (M_k->n != n || A_0->n != n) return SAM_ERR_INVALID_ARG;
    Scratch sc(h);
    Stager sg(sc, h->stream);
    DevCsr a = stage_csr(sg, A_k, true), m = stage_csr(sg, M_k, true), z = stage_csr(sg, A_0, true);
    if (sg.failed) return SAM_ERR_OOM;
    sam_status s = validate_all(h, {a, m, z});
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
    sam_status s = validate_all(h, {m});
    if (s != SAM_OK) return s;
    if (csr_spmv(h, n, m.rp, m.ci, m.v, dx, dy) != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.finish() != cudaSuccess) return SAM_ERR_CUDA;
    if (sg.has_host_outputs()) return drain_status(h);
    return SAM_OK;
}

sam_status sam_build_backward(sam_handle h, const sam_csr *A_k, const sam_csr *A_0, sam_pattern S, int precision,
                              int refine_steps, const double *M_val, const double *dM_val, double *dA_k_val,
                              double *dA_0_val) {
    (void)h; (void)A_k; (void)A_0; (void)S; (void)precision; (void)refine_steps;
    (void)M_val; (void)dM_val; (void)dA_k_val; (void)dA_0_val;
    return SAM_ERR_UNSUPPORTED;
}

sam_status sam_tune(sam_handle h, int K, const sam_csr *A_k, const sam_csr *A_0, const sam_pattern *S, int precision,
                    int refine_steps, const char *cache_path) {
    (void)h; (void)K; (void)A_k; (void)A_0; (void)S; (void)precision; (void)refine_steps; (void)cache_path;
    return SAM_ERR_UNSUPPORTED;
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
