// C ABI of the Ozaki-II emulated GEMM (arXiv 2602.02549): argument checks,
// workspace layout, constant upload and the launch sequence.  The kernels are
// in oz2_kernels.cuh, included here so that one translation unit owns the
// __constant__ tables.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "oz2.h"
#include "oz2_kernels.cuh"

namespace oz2 {
namespace {

constexpr int kMaxDevices = 64;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------------------ per-device state
struct DeviceState {
    bool tables = false;
    bool smem_attr = false;
    int sms = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // buffers replaced by a larger one: kept (not freed) until the process
    // exits, because a call on another stream or host thread may have been
    // handed one of them and not yet enqueued its kernels
    std::vector<void *> retired;
    // tile width per problem of a batch, chosen by oz2_batched_autotune (or set
    // with oz2_batched_set_policy), keyed by the batch's shapes and settings
    std::unordered_map<uint64_t, std::vector<uint8_t>> tiles;
};
std::mutex g_mu;
DeviceState g_dev[kMaxDevices];

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// Last CUDA failure seen by the library (for oz2_last_error): the error code
// and the source line of the check that caught it.
std::atomic<int> g_last_cuda_error{0};
std::atomic<int> g_last_cuda_line{0};

// Kernels launched by the library in this process (oz2_launch_count).
std::atomic<long long> g_launches{0};

int cuda_fail_at(cudaError_t e, int line) {
    if (e == cudaSuccess) return OZ2_OK;
    g_last_cuda_error.store(int(e));
    g_last_cuda_line.store(line);
    (void)cudaGetLastError();
    return OZ2_ECUDA;
}
#define cuda_fail(e) cuda_fail_at((e), __LINE__)

// Upload the host-built tables to this device's constant memory (once).
int ensure_device(int *dev_out) {
    int dev = 0;
    cudaError_t ge = cudaGetDevice(&dev);
    if (ge != cudaSuccess) return cuda_fail(ge);
    if (dev < 0 || dev >= kMaxDevices) return OZ2_ENOTSUP;
    // binds the device's primary context to this host thread: the driver call
    // cuTensorMapEncodeTiled needs a current context, which a thread that has
    // only made runtime calls (e.g. torch's autograd worker) may not have yet
    if ((ge = cudaSetDevice(dev)) != cudaSuccess) return cuda_fail(ge);
    *dev_out = dev;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &st = g_dev[dev];
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return OZ2_ECUDA;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (!st.tables) {
        const Tables &T = tables();
        if (!T.sums_fit) return OZ2_ENOTSUP;
        DevN n64[kNMax + 1], n32[kNMax + 1];
        for (int N = 0; N <= kNMax; N++) {
            const NTable &a = T.n64[N], &b = T.n32[N];
            n64[N] = DevN{a.P1, a.P2, a.Pinv, a.g, a.t, a.gN, a.Pprime, a.eg, a.esum, a.poff,
                          a.M1, a.eu1, a.sh, a.kq, a.sq};
            n32[N] = DevN{b.P1, b.P2, b.Pinv, b.g, b.t, b.gN, b.Pprime, b.eg, b.esum, b.poff,
                          b.M1, b.eu1, b.sh, b.kq, b.sq};
        }
        cudaError_t e = cudaSuccess;
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_n64, n64, sizeof n64);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_n32, n32, sizeof n32);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_dp64, T.dp64, sizeof T.dp64);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_dp32, T.dp32, sizeof T.dp32);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cneg, &T.c, sizeof T.c);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w12, T.mod.w12, sizeof T.mod.w12);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w13p, T.mod.w13p, sizeof T.mod.w13p);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_pf, T.mod.pf, sizeof T.mod.pf);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_invp, T.mod.invp, sizeof T.mod.invp);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_pow2, T.mod.pow2, sizeof T.mod.pow2);
        if (e != cudaSuccess) return cuda_fail(e);
        st.tables = true;
    }
    if (!st.sms) {
        cudaError_t e = cudaDeviceGetAttribute(&st.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (!st.smem_attr) {
        const int s256 = int(gemm::Cfg<256>::kSmemBytes), s128 = int(gemm::Cfg<128>::kSmemBytes);
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaFuncSetAttribute(k_gemm<EPI_MAX, 256, 1>, a, s256);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_MOD, 256, 1>, a, s256);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_MAX, 128, 1>, a, s128);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_MOD, 128, 1>, a, s128);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_MAX, 256, gemm::kMaxGroup>, a, s256);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_MOD, 256, gemm::kMaxGroup>, a, s256);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_MAX, 128, gemm::kMaxGroup>, a, s128);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_MOD, 128, gemm::kMaxGroup>, a, s128);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_CW, 256, 1>, a, s256);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_CW, 128, 1>, a, s128);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_CW, 256, gemm::kMaxGroup>, a, s256);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm<EPI_CW, 128, gemm::kMaxGroup>, a, s128);
        if (e != cudaSuccess) return cuda_fail(e);
        st.smem_attr = true;
    }
    return OZ2_OK;
}

// ------------------------------------------------------------------ workspace layout
struct Dims {
    int m, n, k, m_pad, n_pad, k_pad, nmax;
};

// bn: the GEMM tile width the problem runs with (256 or 128); n is padded to it
Dims make_dims(int m, int n, int k, int nmax, int bn = gemm::kMaxBN) {
    Dims d;
    d.m = m; d.n = n; d.k = k;
    d.m_pad = int(round_up(size_t(m), gemm::BM));
    d.n_pad = int(round_up(size_t(n), size_t(bn)));
    d.k_pad = int(round_up(size_t(k), gemm::BK));
    d.nmax = nmax;
    return d;
}

struct Layout {
    // the block up to zero_end is cleared at the start of every call
    size_t hmaxA, hmaxB, cmax_row, cmax_col, red, ssA, ssB, rmaxA, rmaxB, l1A, l1B, cwA, cwB, zero_end;
    size_t mu, nu, ndev, resA, resB, W, total;
};

Layout make_layout(const Dims &d) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = round_up(o + bytes, 256); return at; };
    L.hmaxA = take(sizeof(unsigned long long) * size_t(d.k_pad));
    L.hmaxB = take(sizeof(unsigned long long) * size_t(d.k_pad));
    L.cmax_row = take(sizeof(int) * size_t(d.m_pad));
    L.cmax_col = take(sizeof(int) * size_t(d.n_pad));
    L.red = take(sizeof(unsigned long long) * 8);
    L.ssA = take(sizeof(int) * size_t(d.m_pad));
    L.ssB = take(sizeof(int) * size_t(d.n_pad));
    L.rmaxA = take(sizeof(unsigned long long) * size_t(d.m_pad));
    L.rmaxB = take(sizeof(unsigned long long) * size_t(d.n_pad));
    L.l1A = take(2 * sizeof(unsigned long long) * size_t(d.m_pad));
    L.l1B = take(2 * sizeof(unsigned long long) * size_t(d.n_pad));
    L.cwA = take(2 * sizeof(float) * size_t(d.m_pad));
    L.cwB = take(2 * sizeof(float) * size_t(d.n_pad));
    L.zero_end = o;
    L.mu = take(sizeof(int32_t) * size_t(d.m_pad));
    L.nu = take(sizeof(int32_t) * size_t(d.n_pad));
    L.ndev = take(sizeof(int) * 4);
    L.resA = take(size_t(2) * size_t(d.nmax) * size_t(d.m_pad) * size_t(d.k_pad));
    L.resB = take(size_t(2) * size_t(d.nmax) * size_t(d.n_pad) * size_t(d.k_pad));
    L.W = take(size_t(d.nmax) * size_t(d.m_pad) * size_t(d.n_pad));
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ tensor maps
int encode_bf16_2d(CUtensorMap *tm, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {uint32_t(gemm::BK), box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        g_last_cuda_error.store(10000 + int(r));   // driver result, offset to tell it apart
        g_last_cuda_line.store(__LINE__);
        return OZ2_ECUDA;
    }
    return OZ2_OK;
}

// Resident blocks of 256 threads per SM of the looping residue kernels (their
// __launch_bounds__ minimum; the transposing one runs twice as many blocks of 128).
constexpr int kResidBlocksPerSM = 3;

// The residue GEMM's failure-path test hook (oz2_gemm_timeout_selftest sets it
// for the duration of one call on its host thread): the k-block whose loads
// each CTA skips on its first item (-1: none) and the limit of every wait.
struct GemmHook {
    int kb = -1;
    unsigned long long limit_ns = kWaitLimitNs;
};
thread_local GemmHook g_hook;

// One persistent launch over the problems of `G` (item counts filled in here):
// one CTA per SM, or fewer when there are fewer work items.
template <int EPI, int BN, int CAP>
int launch_gemm(GemmGroup<CAP> &G, int sms, cudaStream_t st) {
    long long items = 0;
    for (int p = 0; p < G.count; p++) {
        GemmProblem &P = G.p[p];
        P.item_begin = items;
        const long long np = (long long)P.tiles_m * P.tiles_n * P.planes;
        if (np >= (1ll << 31)) return OZ2_ENOTSUP;   // the kernel decodes a problem's items in 32 bits
        items += np;
    }
    G.total_items = items;
    G.wait_limit_ns = EPI == EPI_MOD ? g_hook.limit_ns : kWaitLimitNs;
    G.hook_kb = EPI == EPI_MOD ? g_hook.kb : -1;
    if (items == 0) return OZ2_OK;
    const int grid = int(std::min<long long>(items, sms));
    k_gemm<EPI, BN, CAP><<<grid, gemm::kThreads, gemm::Cfg<BN>::kSmemBytes, st>>>(G);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_fail(cudaGetLastError());
}

// ------------------------------------------------------------------ validation
int validate(int m, int n, int k, const void *A, int lda, const void *B, int ldb, const void *C, int ldc,
             int nmoduli, int mode, const oz2_opts *o) {
    if (m < 1 || n < 1 || k < 1) return OZ2_EINVAL;
    if (!A || !B || !C) return OZ2_EINVAL;
    if (mode & ~(OZ2_FAST | OZ2_TRANS_A | OZ2_TRANS_B | OZ2_COMPONENTWISE)) return OZ2_EINVAL;
    const bool ta = mode & OZ2_TRANS_A, tb = mode & OZ2_TRANS_B;
    if (lda < (ta ? m : k) || ldb < (tb ? k : n) || ldc < n) return OZ2_EINVAL;
    if (nmoduli != 0 && (nmoduli < OZ2_N_MIN || nmoduli > OZ2_N_MAX)) return OZ2_EINVAL;
    if (nmoduli != 0 && (mode & OZ2_COMPONENTWISE)) return OZ2_EINVAL;   // a rule for choosing N
    if (nmoduli == 0) {
        if (!o || !(o->target > 0.0)) return OZ2_EINVAL;
        if (o->nmax != 0 && (o->nmax < OZ2_N_MIN || o->nmax > OZ2_N_MAX)) return OZ2_EINVAL;
    }
    if (o && ((o->mu_in == nullptr) != (o->nu_in == nullptr))) return OZ2_EINVAL;
    if (o && o->mu_in && nmoduli == 0) return OZ2_EINVAL;
    return OZ2_OK;
}

// Split-K beyond the paper's k <= 2^17 (Section 3: the bound that keeps the INT32
// sums of Algorithms 2 and 3 exact): S = ceil(k / 2^17) ranges are wanted; each
// range holds kc = 64 ceil(ceil(k / S) / 64) <= 2^17 consecutive k (the last one
// fewer), so there are count = ceil(k / kc) <= S of them.  k <= 2^17: one range.
struct KSplit {
    int count, kc;
};
inline KSplit k_split(int k) {
    if (k <= OZ2_K_MAX) return KSplit{1, k};
    const long long S = cdiv(k, OZ2_K_MAX);
    const int kc = int(round_up(size_t(cdiv(k, S)), 64));
    return KSplit{int(cdiv(k, kc)), kc};
}

// ------------------------------------------------------------------ the pipeline
// One emulated GEMM, split into the phases that surround the two tensor-core
// GEMMs so that a batch can run the phases of many problems concurrently and
// each GEMM of all problems as one persistent launch.
template <typename T>
struct Job {
    static constexpr bool fp32 = sizeof(T) == 4;
    // arguments
    int m = 0, n = 0, k = 0, lda = 0, ldb = 0, ldc = 0, nmoduli = 0, mode = 0, nmax = 0;
    int bn = gemm::kMaxBN;         // GEMM tile width (n is padded to it)
    const T *A = nullptr, *B = nullptr;
    T *C = nullptr;
    double target = 0.0;
    int *n_out = nullptr;
    int32_t *mu_out = nullptr, *nu_out = nullptr;
    const int32_t *mu_in = nullptr, *nu_in = nullptr;
    bool accum = false;            // CRT adds to C (split-K ranges after the first)
    // workspace views
    Dims d{};
    Layout L{};
    uint8_t *ws = nullptr;
    unsigned long long *hmaxA, *hmaxB, *red, *rmaxA, *rmaxB, *l1A, *l1B;
    float *cwA, *cwB;
    int *cmax_row, *cmax_col, *ssA, *ssB, *ndev;
    int32_t *mu, *nu;
    __nv_bfloat16 *resA, *resB;
    int8_t *W;
    Operand<T> opA{}, opB{};
    long planeA = 0, planeB = 0, w_plane = 0;

    bool fast() const { return mode & OZ2_FAST; }
    bool cw() const { return mode & OZ2_COMPONENTWISE; }
    bool inject() const { return mu_in != nullptr; }
    bool needs_scale_gemm() const { return !fast() && !inject(); }

    void set(int m_, int n_, int k_, const T *A_, int lda_, const T *B_, int ldb_, T *C_, int ldc_, int N_, int mode_,
             double target_, int nmax_, int bn_ = gemm::kMaxBN) {
        m = m_; n = n_; k = k_; A = A_; lda = lda_; B = B_; ldb = ldb_; C = C_; ldc = ldc_;
        nmoduli = N_; mode = mode_; target = target_;
        nmax = N_ ? N_ : (nmax_ ? nmax_ : (fp32 ? 14 : 20));
        bn = bn_;
        d = make_dims(m, n, k, nmax, bn);
        L = make_layout(d);
    }

    void bind(uint8_t *w) {
        ws = w;
        auto at = [&](size_t off) { return ws + off; };
        hmaxA = reinterpret_cast<unsigned long long *>(at(L.hmaxA));
        hmaxB = reinterpret_cast<unsigned long long *>(at(L.hmaxB));
        cmax_row = reinterpret_cast<int *>(at(L.cmax_row));
        cmax_col = reinterpret_cast<int *>(at(L.cmax_col));
        red = reinterpret_cast<unsigned long long *>(at(L.red));
        ssA = reinterpret_cast<int *>(at(L.ssA));
        ssB = reinterpret_cast<int *>(at(L.ssB));
        rmaxA = reinterpret_cast<unsigned long long *>(at(L.rmaxA));
        rmaxB = reinterpret_cast<unsigned long long *>(at(L.rmaxB));
        l1A = reinterpret_cast<unsigned long long *>(at(L.l1A));
        l1B = reinterpret_cast<unsigned long long *>(at(L.l1B));
        cwA = reinterpret_cast<float *>(at(L.cwA));
        cwB = reinterpret_cast<float *>(at(L.cwB));
        mu = reinterpret_cast<int32_t *>(at(L.mu));
        nu = reinterpret_cast<int32_t *>(at(L.nu));
        ndev = reinterpret_cast<int *>(at(L.ndev));
        resA = reinterpret_cast<__nv_bfloat16 *>(at(L.resA));
        resB = reinterpret_cast<__nv_bfloat16 *>(at(L.resB));
        W = reinterpret_cast<int8_t *>(at(L.W));
        const bool ta = mode & OZ2_TRANS_A, tb = mode & OZ2_TRANS_B;
        // A's logical rows are the rows of A; B's are the columns of B.
        opA = Operand<T>{A, long(lda), m, ta ? 0 : 1};
        opB = Operand<T>{B, long(ldb), n, tb ? 1 : 0};
        planeA = long(d.m_pad) * d.k_pad;
        planeB = long(d.n_pad) * d.k_pad;
        w_plane = long(d.m_pad) * d.n_pad;
    }

    const int32_t *mu_use() const { return inject() ? mu_in : mu; }
    const int32_t *nu_use() const { return inject() ? nu_in : nu; }

    // the residue planes and their tensor maps (plane 0 holds Abar / Bbar first)
    // tile width w: the problem's own (bn), or 128 where n_pad is a multiple of 256
    int describe(GemmProblem &P, int w = 0) const {
        if (w == 0) w = bn;
        int rc = encode_bf16_2d(&P.tmA, resA, uint64_t(nmax) * d.m_pad, uint64_t(d.k_pad), gemm::BM);
        if (rc) return rc;
        if ((rc = encode_bf16_2d(&P.tmB, resB, uint64_t(nmax) * d.n_pad, uint64_t(d.k_pad), uint32_t(w)))) return rc;
        P.m_pad = d.m_pad;
        P.n_pad = d.n_pad;
        P.kb_total = d.k_pad / gemm::BK;
        P.tiles_m = d.m_pad / gemm::BM;
        P.tiles_n = d.n_pad / w;
        P.plane0 = 0;
        P.cw_row = P.cw_col = nullptr;
        P.cw_red = nullptr;
        return OZ2_OK;
    }
    void as_scale_gemm(GemmProblem &P) const {
        P.planes = 1;
        P.n_dev = nullptr;
        P.W = nullptr;
        P.row_max = cmax_row;
        P.col_max = cmax_col;
    }
    void as_residue_gemm(GemmProblem &P) const {
        P.planes = nmax;
        P.n_dev = ndev;
        P.W = W;
        P.w_plane = w_plane;
        P.row_max = P.col_max = nullptr;
    }
    // componentwise rule: floor(2^mu' |A|) floor(|B| 2^nu') from plane 1
    void as_cw_gemm(GemmProblem &P) const {
        P.planes = 1;
        P.plane0 = 1;
        P.n_dev = nullptr;
        P.W = nullptr;
        P.row_max = P.col_max = nullptr;
        P.cw_row = cwA;
        P.cw_col = cwB;
        P.cw_red = red + 5;
    }

    // the device view of this problem for the grouped light-phase kernels
    JobDesc<T> desc() const {
        JobDesc<T> j{};
        j.absmax_lb = kLineBlock;
        j.op[0] = opA;
        j.op[1] = opB;
        j.C = C;
        j.ldc = ldc;
        j.m = m; j.n = n; j.k = k;
        j.k_pad = d.k_pad;
        j.n_pad = d.n_pad;
        j.R_pad[0] = d.m_pad;
        j.R_pad[1] = d.n_pad;
        j.nmoduli = nmoduli;
        j.nmax = nmax;
        j.fast = fast() ? 1 : 0;
        j.cw = cw() ? 1 : 0;
        j.cwv[0] = cwA;
        j.cwv[1] = cwB;
        j.inject = inject() ? 1 : 0;
        j.accum = accum ? 1 : 0;
        auto aligned = [](const Operand<T> &op) {
            return (reinterpret_cast<uintptr_t>(op.ptr) % 16 == 0 && (op.ld * long(sizeof(T))) % 16 == 0) ? 1 : 0;
        };
        j.vec[0] = aligned(opA);
        j.vec[1] = aligned(opB);
        j.target = nmoduli ? 0.0 : target;
        j.hmax[0] = hmaxA; j.hmax[1] = hmaxB;
        j.rmax[0] = rmaxA; j.rmax[1] = rmaxB;
        j.l1[0] = l1A; j.l1[1] = l1B;
        j.red = red;
        j.cmax[0] = cmax_row; j.cmax[1] = cmax_col;
        j.ss[0] = ssA; j.ss[1] = ssB;
        j.ndev = ndev;
        j.n_out = n_out;
        j.expo[0] = mu; j.expo[1] = nu;
        j.shift[0] = mu_use(); j.shift[1] = nu_use();
        j.expo_out[0] = mu_out; j.expo_out[1] = nu_out;
        j.res[0] = resA; j.res[1] = resB;
        j.plane[0] = planeA; j.plane[1] = planeB;
        j.W = W;
        j.w_plane = w_plane;
        j.zero = reinterpret_cast<uint4 *>(ws);
        j.zero_vec = long(L.zero_end / 16);
        for (int X = 0; X < 2; X++) {        // run_group may narrow these per launch
            int S, Cl;
            absmax_geom(j, X, S, Cl);
            j.absmax_lw[X] = absmax_lw_min(Cl);
        }
        return j;
    }
};

// The library-managed workspace of the current device, for calls without a
// workspace of their own: one buffer per device, shared by every such call (so
// those calls must not overlap on the GPU).  It grows with cudaMalloc, by at
// least a quarter each time so that the superseded buffers, which stay
// allocated until the process exits, add up to a bounded multiple of the
// largest size.  Nothing synchronises the device or frees memory here.
int managed_workspace(int dev, size_t bytes, uint8_t **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &s = g_dev[dev];
    if (s.ws_bytes < bytes) {
        size_t size = std::max(bytes, s.ws_bytes + s.ws_bytes / 4);
        void *p = nullptr;
        if (cudaMalloc(&p, size) != cudaSuccess) {
            (void)cudaGetLastError();
            size = bytes;                    // the larger step did not fit: exactly what is needed
            if (cudaMalloc(&p, size) != cudaSuccess) return cuda_fail(cudaErrorMemoryAllocation);
        }
        if (s.ws) s.retired.push_back(s.ws);
        s.ws = p;
        s.ws_bytes = size;
    }
    *out = static_cast<uint8_t *>(s.ws);
    return OZ2_OK;
}

// Every phase of Algorithms 1-3 for a group of at most kMaxJobs problems:
// each light phase is one launch over the items of all problems, each GEMM one
// persistent launch over the tiles of all problems (heaviest first).
// part: 0 the whole call; 1 the phases up to the N rule's reductions (a rank's
// share before the exchange of a row-sharded call); 2 the rest, from the
// reductions again (after the exchange)
enum { kPartAll = 0, kPartBegin = 1, kPartEnd = 2 };
template <typename T, int CAP, class Mark>
int run_group(Job<T> *const *jobs, int count, cudaStream_t st, int sms, Mark &&mark, int part = kPartAll) {
    static_assert(sizeof(JobGroup<T, CAP>) < 30000 && sizeof(GemmGroup<CAP>) < 30000, "kernel parameter space");
    static thread_local JobGroup<T, CAP> J;      // passed by value as the kernel parameter
    static thread_local GemmGroup<CAP> G;
    std::memset(&J, 0, sizeof J);
    J.count = count;
    for (int p = 0; p < count; p++) J.j[p] = jobs[p]->desc();
    // k_absmax: items of the width that wastes the fewest positions (absmax_lw_min); while the whole
    // launch would give fewer than two blocks per SM, narrower items (more line
    // groups per block), and then, while it would give fewer than one, fewer
    // lines per item.  Each item ends in one atomicMax per position and per
    // line, and the items that share a position contend for it, so launches
    // with enough items keep the widest items and the full kLineBlock lines.
    {
        auto total = [&]() {
            long long t = 0;
            for (int p = 0; p < count; p++) t += Items<T>::absmax(J.j[p]);
            return t;
        };
        for (bool wider = true; wider && total() < 2ll * sms;) {
            wider = false;
            for (int p = 0; p < count; p++)
                for (int X = 0; X < 2; X++)
                    if (J.j[p].absmax_lw[X] < 8) { J.j[p].absmax_lw[X] *= 2; wider = true; }
        }
        while (total() < sms && J.j[0].absmax_lb > 8)
            for (int p = 0; p < count; p++) J.j[p].absmax_lb /= 2;
    }
    // fills J.begin from the per-problem item counts; returns the grid size (0: nothing to do)
    // (the kernels decode a problem's items with 32-bit arithmetic; a count of
    // 2^32 would need terabytes of workspace, and is refused)
    auto plan = [&](long long (*items)(const JobDesc<T> &), long long cap) -> int {
        J.begin[0] = 0;
        for (int p = 0; p < count; p++) {
            const long long c = items(J.j[p]);
            if (c >= (1ll << 32)) return -1;
            J.begin[p + 1] = J.begin[p] + c;
        }
        return int(std::min<long long>(J.begin[count], cap));
    };
    // one item per block where a block has no setup to amortise; the residue
    // kernels (the per-item N load and plane constants) stay resident and loop,
    // kResidBlocksPerSM blocks of 256 threads per SM (their launch bound)
    const long long one_each = (1ll << 31) - 1, resident = (long long)sms * kResidBlocksPerSM;
    int rc, g;
    auto launched = [&]() { return cuda_fail(cudaGetLastError()); };
#define OZ2_LAUNCH_B(kernel, items, cap, threads)                    \
    if ((g = plan(Items<T>::items, cap)) < 0) return OZ2_ENOTSUP;   \
    if (g > 0) {                                                    \
        kernel<T, CAP><<<g, threads, 0, st>>>(J);                   \
        g_launches.fetch_add(1, std::memory_order_relaxed);         \
        if ((rc = launched())) return rc;                           \
    }
#define OZ2_LAUNCH(kernel, items, cap) OZ2_LAUNCH_B(kernel, items, cap, 256)
    // heaviest problems first: the longest-processing-time order balances the
    // static assignment of GEMM work items to CTAs
    std::vector<int> order;
    order.resize(size_t(count));
    for (int p = 0; p < count; p++) order[p] = p;
    auto cost = [&](int p) {
        const auto &d = jobs[p]->d;
        return double(d.m_pad) * d.n_pad * d.k_pad * (jobs[p]->nmax + 1);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    // one persistent launch per GEMM phase and tile width: EPI_MAX the scaling
    // GEMM, EPI_CW the componentwise rule's second product, EPI_MOD the residues
    // The scaling GEMM (one plane) of a launch with at most half as many 128 x 256
    // tiles as SMs runs on 128 x 128 tiles: twice the CTAs at work, still one
    // round (1024^3: 16 -> 13 us); larger launches keep each problem's width.
    bool narrow_scale = true;
    {
        long long tiles = 0;
        for (int p = 0; p < count; p++)
            if (jobs[p]->needs_scale_gemm())
                tiles += (long long)(jobs[p]->d.m_pad / gemm::BM) * (jobs[p]->d.n_pad / jobs[p]->bn);
        narrow_scale = 2 * tiles <= sms;
    }
    auto width = [&](const Job<T> &job, int epi) { return epi == EPI_MAX && narrow_scale ? 128 : job.bn; };
    auto gemms = [&](int epi) -> int {
        for (int bn : {256, 128}) {
            std::memset(&G, 0, sizeof G);
            for (int idx = 0; idx < count; idx++) {
                const Job<T> &job = *jobs[order[idx]];
                if (width(job, epi) != bn) continue;
                if ((epi == EPI_MAX && !job.needs_scale_gemm()) || (epi == EPI_CW && !job.cw())) continue;
                GemmProblem &P = G.p[G.count++];
                int r = job.describe(P, bn);
                if (r) return r;
                if (epi == EPI_MAX) job.as_scale_gemm(P);
                else if (epi == EPI_CW) job.as_cw_gemm(P);
                else job.as_residue_gemm(P);
            }
            if (!G.count) continue;
            int r;
            if (bn == 256)
                r = epi == EPI_MAX ? launch_gemm<EPI_MAX, 256>(G, sms, st)
                                   : (epi == EPI_CW ? launch_gemm<EPI_CW, 256>(G, sms, st)
                                                    : launch_gemm<EPI_MOD, 256>(G, sms, st));
            else
                r = epi == EPI_MAX ? launch_gemm<EPI_MAX, 128>(G, sms, st)
                                   : (epi == EPI_CW ? launch_gemm<EPI_CW, 128>(G, sms, st)
                                                    : launch_gemm<EPI_MOD, 128>(G, sms, st));
            if (r) return r;
        }
        return OZ2_OK;
    };

    if (part != kPartEnd) {
        if ((rc = mark(OZ2_PHASE_STATS))) return rc;
        OZ2_LAUNCH(k_clear, clear, one_each)
        OZ2_LAUNCH(k_absmax, absmax, one_each)
        if ((rc = mark(OZ2_PHASE_QUANT))) return rc;
        {   // one launch for both layouts where the two would each leave SMs idle
            long long items = 0;
            for (int p = 0; p < count; p++) items += Items<T>::quant(J.j[p]);
            if (items < 4ll * sms) {
                OZ2_LAUNCH(k_quant, quant, one_each)
            } else {
                OZ2_LAUNCH(k_quant_kc, quant_kc, one_each)
                OZ2_LAUNCH(k_quant_rc, quant_rc, one_each)
            }
        }
        OZ2_LAUNCH(k_fast_max, fast_max, one_each)
        OZ2_LAUNCH(k_fast_cmax, fast_cmax, one_each)
        if ((rc = mark(OZ2_PHASE_SCALEGEMM))) return rc;
        if ((rc = gemms(EPI_MAX))) return rc;
    }
    if ((rc = mark(OZ2_PHASE_EXPONENTS))) return rc;
    // after the exchange the reductions run again: their atomic maxima over
    // this rank's rows leave the exchanged maxima in place, and the terms that
    // read the exchanged column maxima and per-k maxima come out global
    OZ2_LAUNCH(k_bound, bound, one_each)
    if (part == kPartBegin) return OZ2_OK;
    if ((rc = gemms(EPI_CW))) return rc;
    OZ2_LAUNCH(k_exponents, exponents, one_each)
    if ((rc = mark(OZ2_PHASE_RESIDUES))) return rc;
    OZ2_LAUNCH(k_resid_kc, resid_kc, resident)
    OZ2_LAUNCH_B(k_resid_rc, resid_rc, 2 * resident, 128)   // 128-thread blocks, twice as many
    if ((rc = mark(OZ2_PHASE_GEMM))) return rc;
    if ((rc = gemms(EPI_MOD))) return rc;
    if ((rc = mark(OZ2_PHASE_CRT))) return rc;
    if (count == 1) {
        const JobDesc<T> &j = J.j[0];
        dim3 grid(unsigned(cdiv(j.n, kCrtCols)), unsigned(std::min(j.m, 65535)));
        k_crt_one<T><<<grid, 256, 0, st>>>(j.W, j.w_plane, long(j.n_pad), j.ndev, j.shift[0], j.shift[1], j.C,
                                             j.ldc, j.m, j.n, j.accum);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if ((rc = launched())) return rc;
    } else {
        OZ2_LAUNCH(k_crt, crt, one_each)
    }
#undef OZ2_LAUNCH
#undef OZ2_LAUNCH_B
    return mark(OZ2_NPHASES);
}

template <typename T>
int run(int m, int n, int k, const T *A, int lda, const T *B, int ldb, T *C, int ldc, int nmoduli, int mode,
        const oz2_opts *o) {
    int rc = validate(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, o);
    if (rc) return rc;
    const KSplit ks = k_split(k);
    if (ks.count > 1 && o && (o->w_out || o->phase_events)) return OZ2_ENOTSUP;
    // the workspace is laid out for the longest K range and reused by each range
    Job<T> job;
    const double target = o ? o->target / ks.count : 0.0;
    job.set(m, n, ks.kc, A, lda, B, ldb, C, ldc, nmoduli, mode, target, o ? o->nmax : 0);
    int dev = 0;
    if ((rc = ensure_device(&dev))) return rc;
    cudaStream_t st = o ? static_cast<cudaStream_t>(o->stream) : nullptr;
    uint8_t *ws = nullptr;
    if (o && o->workspace) {
        if (o->workspace_bytes < job.L.total) return OZ2_ENOMEM;
        if (reinterpret_cast<uintptr_t>(o->workspace) & 255u) return OZ2_EINVAL;
        ws = static_cast<uint8_t *>(o->workspace);
    } else if ((rc = managed_workspace(dev, job.L.total, &ws))) {
        return rc;
    }
    auto mark = [&](int phase) -> int {
        if (!o || !o->phase_events) return OZ2_OK;
        return cuda_fail(cudaEventRecord(static_cast<cudaEvent_t>(o->phase_events[phase]), st));
    };
    // K range s: A[:, k0:k1] B[k0:k1, :] with its own exponents and N (target / S),
    // added into C after the first range
    const bool ta = mode & OZ2_TRANS_A, tb = mode & OZ2_TRANS_B;
    for (int s = 0; s < ks.count; s++) {
        const int k0 = s * ks.kc, kl = std::min(k - k0, ks.kc);
        const T *As = ta ? A + size_t(k0) * size_t(lda) : A + k0;
        const T *Bs = tb ? B + k0 : B + size_t(k0) * size_t(ldb);
        job.set(m, n, kl, As, lda, Bs, ldb, C, ldc, nmoduli, mode, target, o ? o->nmax : 0);
        job.accum = s > 0;
        if (o) {
            job.n_out = o->n_out ? o->n_out + s : nullptr;
            job.mu_out = o->mu_out ? o->mu_out + size_t(s) * m : nullptr;
            job.nu_out = o->nu_out ? o->nu_out + size_t(s) * n : nullptr;
            job.mu_in = o->mu_in ? o->mu_in + size_t(s) * m : nullptr;
            job.nu_in = o->nu_in ? o->nu_in + size_t(s) * n : nullptr;
        }
        job.bind(ws);
        Job<T> *one = &job;
        if ((rc = run_group<T, 1>(&one, 1, st, g_dev[dev].sms, mark))) return rc;
    }
    if (o && o->w_out) {
        // export W_l (test aid): plane l, m x n row-major, from the padded layout
        for (int l = 0; l < job.nmax; l++) {
            rc = cuda_fail(cudaMemcpy2DAsync(o->w_out + size_t(l) * m * n, size_t(n), job.W + size_t(l) * job.w_plane,
                                             size_t(job.d.n_pad), size_t(n), size_t(m), cudaMemcpyDeviceToDevice, st));
            if (rc) return rc;
        }
    }
    return OZ2_OK;
}

// ------------------------------------------------------------------ host arrays
// oz2_gemm_host / oz2_sgemm_host: the device copies of A, B (packed in their
// stored layout) and C, each rounded up to 256 bytes, then the emulation's own
// workspace (laid out as run<T> lays it out for this call).
struct HostSplit {
    size_t a, b, c, inner, total;
};

template <typename T>
HostSplit host_split(int m, int n, int k, int nmax) {
    HostSplit h{};
    h.a = round_up(size_t(m) * size_t(k) * sizeof(T), 256);
    h.b = round_up(size_t(k) * size_t(n) * sizeof(T), 256);
    h.c = round_up(size_t(m) * size_t(n) * sizeof(T), 256);
    h.inner = make_layout(make_dims(m, n, k_split(k).kc, nmax)).total;
    h.total = h.a + h.b + h.c + h.inner;
    return h;
}

template <typename T>
int run_host(int m, int n, int k, const T *A, int lda, const T *B, int ldb, T *C, int ldc, int nmoduli, int mode,
             const oz2_opts *o) {
    int rc = validate(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, o);
    if (rc) return rc;
    // refused by run<T> too, but only after the uploads: refuse before them
    if (k_split(k).count > 1 && o && (o->w_out || o->phase_events)) return OZ2_ENOTSUP;
    const int nmax = nmoduli ? nmoduli : (o && o->nmax ? o->nmax : (sizeof(T) == 4 ? 14 : 20));
    const HostSplit h = host_split<T>(m, n, k, nmax);
    int dev = 0;
    if ((rc = ensure_device(&dev))) return rc;
    cudaStream_t st = o ? static_cast<cudaStream_t>(o->stream) : nullptr;
    uint8_t *ws = nullptr;
    if (o && o->workspace) {
        if (o->workspace_bytes < h.total) return OZ2_ENOMEM;
        if (reinterpret_cast<uintptr_t>(o->workspace) & 255u) return OZ2_EINVAL;
        ws = static_cast<uint8_t *>(o->workspace);
    } else if ((rc = managed_workspace(dev, h.total, &ws))) {
        return rc;
    }
    const bool ta = mode & OZ2_TRANS_A, tb = mode & OZ2_TRANS_B;
    const int ra = ta ? k : m, ca = ta ? m : k;     // A as stored: ra rows of ca
    const int rb = tb ? n : k, cb = tb ? k : n;     // B likewise
    T *dA = reinterpret_cast<T *>(ws), *dB = reinterpret_cast<T *>(ws + h.a);
    T *dC = reinterpret_cast<T *>(ws + h.a + h.b);
    // cudaMemcpyDefault: the runtime tells host from device memory (unified addressing)
    if ((rc = cuda_fail(cudaMemcpy2DAsync(dA, size_t(ca) * sizeof(T), A, size_t(lda) * sizeof(T),
                                          size_t(ca) * sizeof(T), size_t(ra), cudaMemcpyDefault, st))))
        return rc;
    if ((rc = cuda_fail(cudaMemcpy2DAsync(dB, size_t(cb) * sizeof(T), B, size_t(ldb) * sizeof(T),
                                          size_t(cb) * sizeof(T), size_t(rb), cudaMemcpyDefault, st))))
        return rc;
    oz2_opts inner = o ? *o : oz2_opts{};
    inner.stream = st;
    inner.workspace = ws + h.a + h.b + h.c;
    inner.workspace_bytes = h.inner;
    if ((rc = run<T>(m, n, k, dA, ca, dB, cb, dC, n, nmoduli, mode, &inner))) return rc;
    return cuda_fail(cudaMemcpy2DAsync(C, size_t(ldc) * sizeof(T), dC, size_t(n) * sizeof(T), size_t(n) * sizeof(T),
                                       size_t(m), cudaMemcpyDefault, st));
}

// ------------------------------------------------------------------ complex
// ZGEMM / CGEMM: op(A) op(B) for interleaved complex A, B, C as two real
// emulations over 2k (k_zsplit): Re C = A_s B_1, Im C = A_s B_2 with
// A_s = [Re op(A), Im op(A)], B_1 = [Re op(B); -Im op(B)], B_2 = [Im op(B); Re op(B)].
// Transposed operands stay transposed: their real forms are built transposed
// and handed to the real path with the same OZ2_TRANS_* flag.
struct ZLayout {
    size_t As, B1, B2, Cre, Cim, real, total;
};

template <typename T>
ZLayout zlayout(int m, int n, int k, int nmax, int mode) {
    ZLayout z{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = round_up(o + bytes, 256); return at; };
    const size_t k2 = 2 * size_t(k);
    z.As = take(sizeof(T) * size_t(m) * k2);
    z.B1 = take(sizeof(T) * k2 * size_t(n));
    z.B2 = take(sizeof(T) * k2 * size_t(n));
    z.Cre = take(sizeof(T) * size_t(m) * size_t(n));
    z.Cim = take(sizeof(T) * size_t(m) * size_t(n));
    const size_t real = oz2_workspace_size(m, n, int(k2), nmax, mode, sizeof(T) == 4);
    z.real = take(real);
    z.total = real ? o : 0;
    return z;
}

int zvalidate(int m, int n, int k, const void *A, int lda, const void *B, int ldb, const void *C, int ldc,
              int nmoduli, int mode, const oz2_opts *o, size_t esize) {
    if (m < 1 || n < 1 || k < 1 || k > (1 << 30)) return OZ2_EINVAL;
    if (!A || !B || !C) return OZ2_EINVAL;
    if (mode & ~(OZ2_FAST | OZ2_TRANS_A | OZ2_TRANS_B | OZ2_CONJ_A | OZ2_CONJ_B | OZ2_COMPONENTWISE)) return OZ2_EINVAL;
    const bool ta = mode & OZ2_TRANS_A, tb = mode & OZ2_TRANS_B;
    if (lda < (ta ? m : k) || ldb < (tb ? k : n) || ldc < n) return OZ2_EINVAL;
    const size_t al = 2 * esize;
    if (reinterpret_cast<uintptr_t>(A) % al || reinterpret_cast<uintptr_t>(B) % al ||
        reinterpret_cast<uintptr_t>(C) % al)
        return OZ2_EINVAL;
    if (nmoduli != 0 && (nmoduli < OZ2_N_MIN || nmoduli > OZ2_N_MAX)) return OZ2_EINVAL;
    if (nmoduli == 0) {
        if (!o || !(o->target > 0.0)) return OZ2_EINVAL;
        if (o->nmax != 0 && (o->nmax < OZ2_N_MIN || o->nmax > OZ2_N_MAX)) return OZ2_EINVAL;
    }
    if (o && ((o->mu_in == nullptr) != (o->nu_in == nullptr))) return OZ2_EINVAL;
    if (o && o->mu_in && nmoduli == 0) return OZ2_EINVAL;
    if (o && (o->w_out || o->phase_events)) return OZ2_ENOTSUP;
    return OZ2_OK;
}

template <typename T>
int run_complex(int m, int n, int k, const T *A, int lda, const T *B, int ldb, T *C, int ldc, int nmoduli,
                int mode, const oz2_opts *o) {
    int rc = zvalidate(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, o, sizeof(T));
    if (rc) return rc;
    const bool fp32 = sizeof(T) == 4;
    const int nmax = nmoduli ? nmoduli : (o && o->nmax ? o->nmax : (fp32 ? 14 : 20));
    const int rmode = mode & (OZ2_FAST | OZ2_TRANS_A | OZ2_TRANS_B | OZ2_COMPONENTWISE);
    const ZLayout z = zlayout<T>(m, n, k, nmax, rmode);
    if (!z.total) return OZ2_EINVAL;
    int dev = 0;
    if ((rc = ensure_device(&dev))) return rc;
    cudaStream_t st = o ? static_cast<cudaStream_t>(o->stream) : nullptr;
    uint8_t *ws = nullptr;
    if (o && o->workspace) {
        if (o->workspace_bytes < z.total) return OZ2_ENOMEM;
        if (reinterpret_cast<uintptr_t>(o->workspace) & 255u) return OZ2_EINVAL;
        ws = static_cast<uint8_t *>(o->workspace);
    } else if ((rc = managed_workspace(dev, z.total, &ws))) {
        return rc;
    }
    const bool ta = mode & OZ2_TRANS_A, tb = mode & OZ2_TRANS_B;
    const int ca = (mode & OZ2_CONJ_A) ? 1 : 0, cb = (mode & OZ2_CONJ_B) ? 1 : 0;
    T *As = reinterpret_cast<T *>(ws + z.As), *B1 = reinterpret_cast<T *>(ws + z.B1);
    T *B2 = reinterpret_cast<T *>(ws + z.B2), *Cre = reinterpret_cast<T *>(ws + z.Cre);
    T *Cim = reinterpret_cast<T *>(ws + z.Cim);
    const int k2 = 2 * k;
    auto split = [&](const T *X, int ldx, int R, int L, bool stacked, int im0, int neg0, int im1, int neg1, T *Y,
                     int ldy) {
        dim3 grid(unsigned(cdiv(L, 256)), unsigned(std::min(R, 65535)));
        k_zsplit<T><<<grid, 256, 0, st>>>(X, ldx, R, L, stacked ? 1 : 0, im0, neg0, im1, neg1, Y, ldy);
        g_launches.fetch_add(1, std::memory_order_relaxed);
        return cuda_fail(cudaGetLastError());
    };
    // A_s: m x 2k side by side, or (transposed) 2k x m stacked
    if ((rc = split(A, lda, ta ? k : m, ta ? m : k, ta, 0, 0, 1, ca, As, ta ? m : k2))) return rc;
    // B_1 = [Re; -Im op(B)] and B_2 = [Im op(B); Re]: 2k x n stacked, or (transposed) n x 2k side by side
    const int RB = tb ? n : k, LB = tb ? k : n, ldbs = tb ? k2 : n;
    if ((rc = split(B, ldb, RB, LB, !tb, 0, 0, 1, cb ? 0 : 1, B1, ldbs))) return rc;
    if ((rc = split(B, ldb, RB, LB, !tb, 1, cb, 0, 0, B2, ldbs))) return rc;
    // the two real emulations, one after the other in the shared real workspace
    const int S = k_split(k2).count;
    for (int part = 0; part < 2; part++) {
        oz2_opts r{};
        r.stream = st;
        r.workspace = ws + z.real;
        r.workspace_bytes = z.total - z.real;
        r.target = o ? o->target : 0.0;
        r.nmax = o ? o->nmax : 0;
        if (o) {
            r.n_out = o->n_out ? o->n_out + size_t(part) * S : nullptr;
            r.mu_out = o->mu_out ? o->mu_out + size_t(part) * S * m : nullptr;
            r.nu_out = o->nu_out ? o->nu_out + size_t(part) * S * n : nullptr;
            r.mu_in = o->mu_in ? o->mu_in + size_t(part) * S * m : nullptr;
            r.nu_in = o->nu_in ? o->nu_in + size_t(part) * S * n : nullptr;
        }
        if ((rc = run<T>(m, n, k2, As, ta ? m : k2, part ? B2 : B1, ldbs, part ? Cim : Cre, n, nmoduli, rmode, &r)))
            return rc;
    }
    dim3 grid(unsigned(cdiv(n, 256)), unsigned(std::min(m, 65535)));
    k_zmerge<T><<<grid, 256, 0, st>>>(Cre, Cim, n, m, n, C, ldc);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_fail(cudaGetLastError());
}

// ------------------------------------------------------------------ row-sharded calls
// One rank's rows of a product whose A rows are split over ranks (B whole on
// every rank): the phases up to the N rule's reductions, the exchange (by the
// caller: an element-wise MAX over the ranks of three workspace arrays), then
// the rest.  Algorithm 2's mu_i needs only row i; nu_j needs max_h cbar_hj over
// all rows (the exchanged column maxima), and the bound rule the maxima over
// all rows of |A| v and 2^alpha' and the per-k maxima of |A| (for L).
int rows_check(int m, int n, int k, const double *A, int lda, const double *B, int ldb, int nmoduli, int mode,
               const oz2_opts *o) {
    int rc = validate(m, n, k, A, lda, B, ldb, B, n, nmoduli, mode, o);
    if (rc) return rc;
    if (!o || !o->workspace) return OZ2_EINVAL;                 // the state between the two calls
    if (k > OZ2_K_MAX) return OZ2_ERANGE;
    if ((mode & (OZ2_FAST | OZ2_COMPONENTWISE)) || o->mu_in || o->w_out || o->phase_events) return OZ2_ENOTSUP;
    return OZ2_OK;
}

int rows_part(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
              int nmoduli, int mode, const oz2_opts *o, int part, oz2_exchange *ex) {
    Job<double> job;
    job.set(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, o->target, o->nmax);
    if (o->workspace_bytes < job.L.total) return OZ2_ENOMEM;
    if (reinterpret_cast<uintptr_t>(o->workspace) & 255u) return OZ2_EINVAL;
    int dev = 0, rc = ensure_device(&dev);
    if (rc) return rc;
    job.n_out = o->n_out;
    job.mu_out = o->mu_out;
    job.nu_out = o->nu_out;
    job.bind(static_cast<uint8_t *>(o->workspace));
    if (ex) {
        ex->cmax_col = job.cmax_col;
        ex->n = size_t(n);
        ex->kmax = reinterpret_cast<int64_t *>(job.hmaxA);
        ex->k = size_t(k);
        ex->red = reinterpret_cast<int64_t *>(job.red);
        ex->nred = 8;
    }
    Job<double> *one = &job;
    return run_group<double, 1>(&one, 1, static_cast<cudaStream_t>(o->stream), g_dev[dev].sms,
                                [](int) { return OZ2_OK; }, part);
}

// ------------------------------------------------------------------ batches
int validate_problem(const oz2_problem &q) {
    oz2_opts o{};
    o.target = q.target;
    o.nmax = q.nmax;
    const int rc = validate(q.m, q.n, q.k, q.A, q.lda, q.B, q.ldb, q.C, q.ldc, q.nmoduli, q.mode, &o);
    if (rc) return rc;
    return q.k > OZ2_K_MAX ? OZ2_ERANGE : OZ2_OK;   // no split-K inside a batch
}

// workspace offsets of each problem inside one batch workspace (bn: tile width
// per problem, or null for the widest, which gives the largest layout)
size_t batch_layout(int count, const oz2_problem *q, std::vector<Job<double>> &jobs, std::vector<size_t> &off,
                    const std::vector<uint8_t> *bn = nullptr) {
    jobs.resize(size_t(count));
    off.resize(size_t(count));
    size_t total = 0;
    for (int p = 0; p < count; p++) {
        const int w = bn ? ((*bn)[size_t(p)] ? 128 : 256) : gemm::kMaxBN;
        jobs[p].set(q[p].m, q[p].n, q[p].k, q[p].A, q[p].lda, q[p].B, q[p].ldb, q[p].C, q[p].ldc, q[p].nmoduli,
                    q[p].mode, q[p].target, q[p].nmax, w);
        jobs[p].n_out = q[p].n_out;
        off[p] = total;
        total = round_up(total + jobs[p].L.total, 256);
    }
    return total;
}

// Identity of a batch for the tile cache: every shape and setting of every problem.
uint64_t batch_key(int count, const oz2_problem *q) {
    uint64_t h = 1469598103934665603ull;               // FNV-1a over 64-bit words
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; i++) { h ^= (v >> (8 * i)) & 255u; h *= 1099511628211ull; }
    };
    mix(uint64_t(count));
    for (int p = 0; p < count; p++) {
        uint64_t t;
        std::memcpy(&t, &q[p].target, 8);
        mix(uint64_t(uint32_t(q[p].m)) | (uint64_t(uint32_t(q[p].n)) << 32));
        mix(uint64_t(uint32_t(q[p].k)) | (uint64_t(uint32_t(q[p].nmoduli)) << 32));
        mix(uint64_t(uint32_t(q[p].nmax)) | (uint64_t(uint32_t(q[p].mode)) << 32));
        mix(t);
    }
    return h;
}

// Tile-width policies (entry p: 1 = width 128, 0 = width 256).
constexpr int kPolicies = 4;   // 0 all 256, 1 all 128, 2 narrow ones 128, 3 measured per problem
std::vector<uint8_t> policy_tiles(int policy, int count, const oz2_problem *q) {
    std::vector<uint8_t> t;
    t.resize(size_t(count));
    for (int p = 0; p < count; p++) {
        const int r = q[p].n % 256;
        t[size_t(p)] = policy == 1 ? 1 : (policy == 2 ? uint8_t(r > 0 && r <= 128) : 0);
    }
    return t;
}

int run_batched(int count, const oz2_problem *q, const oz2_opts *o) {
    if (count < 0 || (count > 0 && !q)) return OZ2_EINVAL;
    if (count == 0) return OZ2_OK;
    int rc;
    for (int p = 0; p < count; p++)
        if ((rc = validate_problem(q[p]))) return rc;
    int dev = 0;
    if ((rc = ensure_device(&dev))) return rc;
    std::vector<uint8_t> tiles;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_dev[dev].tiles.find(batch_key(count, q));
        if (it != g_dev[dev].tiles.end() && int(it->second.size()) == count) tiles = it->second;
    }
    std::vector<Job<double>> jobs;
    std::vector<size_t> off;
    const size_t total = batch_layout(count, q, jobs, off, tiles.empty() ? nullptr : &tiles);
    cudaStream_t st = o ? static_cast<cudaStream_t>(o->stream) : nullptr;
    uint8_t *ws = nullptr;
    if (o && o->workspace) {
        if (o->workspace_bytes < total) return OZ2_ENOMEM;
        if (reinterpret_cast<uintptr_t>(o->workspace) & 255u) return OZ2_EINVAL;
        ws = static_cast<uint8_t *>(o->workspace);
    } else if ((rc = managed_workspace(dev, total, &ws))) {
        return rc;
    }
    for (int p = 0; p < count; p++) jobs[p].bind(ws + off[p]);
    std::vector<Job<double> *> ptrs;
    ptrs.resize(size_t(count));
    for (int p = 0; p < count; p++) ptrs[p] = &jobs[p];
    auto mark = [&](int phase) -> int {
        if (!o || !o->phase_events) return OZ2_OK;
        return cuda_fail(cudaEventRecord(static_cast<cudaEvent_t>(o->phase_events[phase]), st));
    };
    auto no_mark = [](int) { return OZ2_OK; };
    const int sms = g_dev[dev].sms;
    // groups of kMaxJobs problems, one after another (phase events: first group)
    for (int first = 0; first < count; first += kMaxJobs) {
        const int c = std::min(kMaxJobs, count - first);
        rc = first == 0 ? run_group<double, kMaxJobs>(ptrs.data(), c, st, sms, mark)
                        : run_group<double, kMaxJobs>(ptrs.data() + first, c, st, sms, no_mark);
        if (rc) return rc;
    }
    return OZ2_OK;
}

// Times each tile policy on this batch (inputs as given, on the caller's
// stream, synchronising) and keeps the fastest for later oz2_gemm_batched
// calls with the same shapes.  Policy 3 first times every problem alone with
// both tile widths and keeps the faster width per problem.
int autotune_batched(int count, const oz2_problem *q, const oz2_opts *o, int *policy_out, float *ms_out) {
    if (count <= 0 || !q) return OZ2_EINVAL;
    int rc;
    for (int p = 0; p < count; p++)
        if ((rc = validate_problem(q[p]))) return rc;
    int dev = 0;
    if ((rc = ensure_device(&dev))) return rc;
    oz2_opts oo{};
    if (o) oo = *o;
    oo.phase_events = nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(oo.stream);
    std::vector<Job<double>> jobs;
    std::vector<size_t> off;
    const size_t need = batch_layout(count, q, jobs, off);
    if (!oo.workspace) {
        uint8_t *ws = nullptr;
        if ((rc = managed_workspace(dev, need, &ws))) return rc;
        oo.workspace = ws;
        oo.workspace_bytes = need;
    } else if (oo.workspace_bytes < need) {
        return OZ2_ENOMEM;
    }
    const uint64_t key = batch_key(count, q);
    auto set_tiles = [&](const std::vector<uint8_t> &t) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_dev[dev].tiles[key] = t;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = cuda_fail(cudaEventCreate(&e0))) || (rc = cuda_fail(cudaEventCreate(&e1)))) return rc;
    // milliseconds per call of fn (one warm-up, then `reps` timed)
    auto timed = [&](auto &&fn, int reps, float *ms) -> int {
        int r = fn();
        if (r) return r;
        if ((r = cuda_fail(cudaEventRecord(e0, st)))) return r;
        for (int i = 0; i < reps && !r; i++) r = fn();
        if (r) return r;
        if ((r = cuda_fail(cudaEventRecord(e1, st)))) return r;
        if ((r = cuda_fail(cudaEventSynchronize(e1)))) return r;
        float t = 0.0f;
        if ((r = cuda_fail(cudaEventElapsedTime(&t, e0, e1)))) return r;
        *ms = t / float(reps);
        return OZ2_OK;
    };
    float ms[kPolicies] = {0, 0, 0, 0};
    std::vector<uint8_t> best_tiles;
    int best = -1;
    for (int pol = 0; pol < kPolicies && !rc; pol++) {
        std::vector<uint8_t> t;
        if (pol < 3) {
            t = policy_tiles(pol, count, q);
        } else {
            // each problem alone, with each width, in its own slice of the workspace
            t.resize(size_t(count));
            for (int p = 0; p < count && !rc; p++) {
                float w[2] = {0, 0};
                for (int wi = 0; wi < 2 && !rc; wi++) {
                    Job<double> job;
                    job.set(q[p].m, q[p].n, q[p].k, q[p].A, q[p].lda, q[p].B, q[p].ldb, q[p].C, q[p].ldc,
                            q[p].nmoduli, q[p].mode, q[p].target, q[p].nmax, wi ? 128 : 256);
                    job.n_out = q[p].n_out;
                    job.bind(static_cast<uint8_t *>(oo.workspace) + off[size_t(p)]);
                    Job<double> *one = &job;
                    auto fn = [&]() {
                        return run_group<double, 1>(&one, 1, st, g_dev[dev].sms, [](int) { return OZ2_OK; });
                    };
                    rc = timed(fn, 2, &w[wi]);
                }
                t[size_t(p)] = w[1] < w[0] ? 1 : 0;
            }
            if (rc) break;
        }
        set_tiles(t);
        auto fn = [&]() { return run_batched(count, q, &oo); };
        if ((rc = timed(fn, 3, &ms[pol]))) break;
        if (best < 0 || ms[pol] < ms[best]) { best = pol; best_tiles = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    set_tiles(best_tiles);
    if (policy_out) *policy_out = best;
    if (ms_out)
        for (int i = 0; i < kPolicies; i++) ms_out[i] = ms[i];
    return OZ2_OK;
}

int set_batched_policy(int count, const oz2_problem *q, int policy) {
    if (count <= 0 || !q || policy < 0 || policy > 2) return OZ2_EINVAL;
    int dev = 0, rc = ensure_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    g_dev[dev].tiles[batch_key(count, q)] = policy_tiles(policy, count, q);
    return OZ2_OK;
}

}  // namespace
}  // namespace oz2

using namespace oz2;

extern "C" {

int oz2_gemm_ex(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
                int nmoduli, int mode, const oz2_opts *opts) {
    return run<double>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, opts);
}

int oz2_gemm(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
             int nmoduli, int mode) {
    return run<double>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, nullptr);
}

int oz2_sgemm_ex(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                 int nmoduli, int mode, const oz2_opts *opts) {
    return run<float>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, opts);
}

int oz2_gemm_host(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
                  int nmoduli, int mode, const oz2_opts *opts) {
    return run_host<double>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, opts);
}

int oz2_sgemm_host(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
                   int nmoduli, int mode, const oz2_opts *opts) {
    return run_host<float>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, opts);
}

size_t oz2_host_workspace_size(int m, int n, int k, int nmax, int mode, int fp32) {
    (void)mode;
    if (m < 1 || n < 1 || k < 1 || nmax < OZ2_N_MIN || nmax > OZ2_N_MAX) return 0;
    return fp32 ? host_split<float>(m, n, k, nmax).total : host_split<double>(m, n, k, nmax).total;
}

int oz2_sgemm(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
              int nmoduli, int mode) {
    return run<float>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, nullptr);
}

int oz2_zgemm(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
              int nmoduli, int mode, const oz2_opts *opts) {
    return run_complex<double>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, opts);
}

int oz2_cgemm(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C, int ldc,
              int nmoduli, int mode, const oz2_opts *opts) {
    return run_complex<float>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, opts);
}

size_t oz2_zworkspace_size(int m, int n, int k, int nmax, int mode, int fp32) {
    if (m < 1 || n < 1 || k < 1 || k > (1 << 30) || nmax < OZ2_N_MIN || nmax > OZ2_N_MAX) return 0;
    const int rmode = mode & (OZ2_FAST | OZ2_TRANS_A | OZ2_TRANS_B | OZ2_COMPONENTWISE);
    return fp32 ? zlayout<float>(m, n, k, nmax, rmode).total : zlayout<double>(m, n, k, nmax, rmode).total;
}

int oz2_gemm_rows_begin(int m, int n, int k, const double *A, int lda, const double *B, int ldb, int nmoduli,
                        int mode, const oz2_opts *opts, oz2_exchange *ex) {
    if (!ex) return OZ2_EINVAL;
    int rc = rows_check(m, n, k, A, lda, B, ldb, nmoduli, mode, opts);
    if (rc) return rc;
    return rows_part(m, n, k, A, lda, B, ldb, nullptr, n, nmoduli, mode, opts, kPartBegin, ex);
}

int oz2_gemm_rows_end(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
                      int nmoduli, int mode, const oz2_opts *opts) {
    int rc = rows_check(m, n, k, A, lda, B, ldb, nmoduli, mode, opts);
    if (rc) return rc;
    if (!C || ldc < n) return OZ2_EINVAL;
    return rows_part(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, mode, opts, kPartEnd, nullptr);
}

int oz2_gemm_batched(int count, const oz2_problem *problems, const oz2_opts *opts) {
    return run_batched(count, problems, opts);
}

int oz2_batched_autotune(int count, const oz2_problem *problems, const oz2_opts *opts, int *policy,
                         float *ms) {
    return autotune_batched(count, problems, opts, policy, ms);
}

int oz2_batched_set_policy(int count, const oz2_problem *problems, int policy) {
    return set_batched_policy(count, problems, policy);
}

size_t oz2_batched_workspace_size(int count, const oz2_problem *problems) {
    if (count < 0 || (count > 0 && !problems)) return 0;
    for (int p = 0; p < count; p++) {
        const oz2_problem &q = problems[p];
        if (q.m < 1 || q.n < 1 || q.k < 1 || q.k > OZ2_K_MAX) return 0;
        if (q.nmoduli != 0 && (q.nmoduli < OZ2_N_MIN || q.nmoduli > OZ2_N_MAX)) return 0;
        if (q.nmax != 0 && (q.nmax < OZ2_N_MIN || q.nmax > OZ2_N_MAX)) return 0;
    }
    std::vector<Job<double>> jobs;
    std::vector<size_t> off;
    return batch_layout(count, problems, jobs, off);
}

size_t oz2_workspace_size(int m, int n, int k, int nmax, int mode, int fp32) {
    (void)mode;
    (void)fp32;
    if (m < 1 || n < 1 || k < 1 || nmax < OZ2_N_MIN || nmax > OZ2_N_MAX) return 0;
    return make_layout(make_dims(m, n, k_split(k).kc, nmax)).total;
}

int oz2_k_ranges(int k, int *count, int *kc) {
    if (k < 1 || !count || !kc) return OZ2_EINVAL;
    const KSplit s = k_split(k);
    *count = s.count;
    *kc = s.kc;
    return OZ2_OK;
}

int oz2_sync(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e);
    int s = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&s, g_status, sizeof s) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    if (s) {
        if (cudaMemcpyToSymbol(g_status, &zero, sizeof zero) != cudaSuccess) return cuda_fail(cudaErrorUnknown);
        return OZ2_ETIMEOUT;
    }
    return OZ2_OK;
}

int oz2_tables(int N, int fp32, double *s1, double *s2, double *scal, float *pprime) {
    if (N < OZ2_N_MIN || N > OZ2_N_MAX || !s1 || !s2 || !scal || !pprime) return OZ2_EINVAL;
    const Tables &T = tables();
    const NTable &t = fp32 ? T.n32[N] : T.n64[N];
    for (int l = 0; l < N; l++) {
        s1[l] = fp32 ? T.s1f[t.offset + l] : T.s1d[t.offset + l];
        s2[l] = fp32 ? 0.0 : T.s2d[t.offset + l];
    }
    scal[0] = t.P1;
    scal[1] = t.P2;
    scal[2] = t.Pinv;
    scal[3] = fp32 ? 0.0 : t.g;
    scal[4] = t.t;
    scal[5] = t.gN;
    *pprime = t.Pprime;
    return OZ2_OK;
}

int oz2_sum_tables(int N, int fp32, int *k, int *esum) {
    if (N < OZ2_N_MIN || N > OZ2_N_MAX || !k || !esum) return OZ2_EINVAL;
    const Tables &T = tables();
    if (!T.sums_fit) return OZ2_ENOTSUP;
    const NTable &t = fp32 ? T.n32[N] : T.n64[N];
    const int(*src)[2] = fp32 ? T.ks32 : T.ks64;
    for (int l = 0; l < N; l++) {
        k[2 * l] = src[t.offset + l][0];
        k[2 * l + 1] = src[t.offset + l][1];
    }
    *esum = t.esum;
    return OZ2_OK;
}

int oz2_check_log2f(void *stream, unsigned long long *dev_out) {
    if (!dev_out) return OZ2_EINVAL;
    int dev = 0, rc = ensure_device(&dev);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float lo = 1.0f, hi = 536870912.0f;   // 2^29
    uint32_t b0, b1;
    std::memcpy(&b0, &lo, 4);
    std::memcpy(&b1, &hi, 4);
    rc = cuda_fail(cudaMemsetAsync(dev_out, 0, 2 * sizeof(unsigned long long), st));
    if (rc) return rc;
    k_log2f_check<<<148 * 8, 256, 0, st>>>(b0, b1 - b0 + 1, dev_out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_fail(cudaGetLastError());
}

int oz2_wait_selftest(void *stream, unsigned int limit_us) {
    if (limit_us == 0 || limit_us > 1000000u) return OZ2_EINVAL;
    int dev = 0, rc = ensure_device(&dev);
    if (rc) return rc;
    k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(uint64_t(limit_us) * 1000ull);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_fail(cudaGetLastError());
}

int oz2_gemm_timeout_selftest(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C,
                              int ldc, int nmoduli, unsigned int limit_us, const oz2_opts *opts) {
    if (limit_us == 0 || limit_us > 1000000u || k <= gemm::BK || k > OZ2_K_MAX) return OZ2_EINVAL;
    g_hook.kb = 1;
    g_hook.limit_ns = (unsigned long long)limit_us * 1000ull;
    const int rc = run<double>(m, n, k, A, lda, B, ldb, C, ldc, nmoduli, 0, opts);
    g_hook = GemmHook{};
    return rc;
}

int oz2_last_error(int *line) {
    if (line) *line = g_last_cuda_line.load();
    return g_last_cuda_error.load();
}

const char *oz2_status_str(int s) {
    switch (s) {
    case OZ2_OK: return "OZ2_OK";
    case OZ2_EINVAL: return "OZ2_EINVAL: invalid argument";
    case OZ2_ERANGE: return "OZ2_ERANGE: k exceeds 2^17 in a batched problem";
    case OZ2_ENOMEM: return "OZ2_ENOMEM: workspace too small";
    case OZ2_ECUDA: return "OZ2_ECUDA: CUDA call failed";
    case OZ2_ETIMEOUT: return "OZ2_ETIMEOUT: a device-side wait gave up";
    case OZ2_ENOTSUP: return "OZ2_ENOTSUP: not supported";
    default: return "unknown status";
    }
}

long long oz2_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int oz2_version(void) { return 100; }

}  // extern "C"
