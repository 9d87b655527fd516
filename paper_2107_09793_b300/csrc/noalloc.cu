// Allocation-free pairwise contraction (jet_pair_contract_noalloc).
//
// For callers that must not allocate device memory: a serving process whose
// GPU memory is pre-reserved by its own allocator (a cudaMalloc behind its back
// can fail or fragment that pool), or a latency-critical loop where cudaMalloc /
// cudaFree would add implicit device synchronisation.  The caller passes device
// inputs and a device output; the split-K partial sums and the offset tables
// live in one fixed, file-scope device array instead of the plan workspace.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <unordered_set>
#include <vector>

#include "internal.h"
#include "kernel_args.h"
#include "kernels.cuh"

namespace jet {

// Fixed scratch shared by every call on a device: [0, 64 KiB) holds the offset
// tables and the three address slots, the rest holds the split-K partials.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;
constexpr size_t NOALLOC_TABLE_BYTES = (size_t)64 << 10;
constexpr int64_t NOALLOC_MAX_OUT = (int64_t)65535 * JET_SPLITK_G;   // output groups fit one grid dimension
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256] = {nullptr};

// Device address of the scratch array on `device` (the array's name is only a
// host-side stand-in).  Looked up once per device, with that device current.
static void *noalloc_scratch_address(int device)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (device < 0 || device >= 256) fail(JET_EINVAL, "device ordinal out of range");
    if (!g_noalloc_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(JET_ECUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") + cudaGetErrorString(e));
        }
        g_noalloc_addr[device] = p;
    }
    return g_noalloc_addr[device];
}

static void check(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(JET_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

void pair_contract_noalloc(int32_t rank_a, const int64_t *labels_a, const int32_t *dims_a, const void *a_dev,
                           int32_t rank_b, const int64_t *labels_b, const int32_t *dims_b, const void *b_dev,
                           void *c_dev, int32_t device, void *stream)
{
    if (!a_dev || !b_dev || !c_dev) fail(JET_EINVAL, "NULL tensor pointer");
    if (rank_a < 0 || rank_b < 0 || rank_a > JET_MAXR || rank_b > JET_MAXR)
        fail(JET_EINVAL, "rank out of range (0.." + std::to_string(JET_MAXR) + ")");
    if ((rank_a && (!labels_a || !dims_a)) || (rank_b && (!labels_b || !dims_b))) fail(JET_EINVAL, "NULL labels/dims");
    // labels, dims and strides of both operands (row-major, labels[0] slowest)
    struct Op1 {
        std::vector<int64_t> l, d, s;
    } A, B;
    auto load = [](Op1 &o, int32_t r, const int64_t *l, const int32_t *d) {
        std::unordered_set<int64_t> seen;
        for (int32_t i = 0; i < r; ++i) {
            if (d[i] < 1) fail(JET_EINVAL, "dim < 1");
            if (!seen.insert(l[i]).second) fail(JET_EINVAL, "label repeated within a tensor");
            o.l.push_back(l[i]);
            o.d.push_back(d[i]);
        }
        o.s.assign(r, 1);
        for (int32_t i = r - 2; i >= 0; --i) o.s[i] = o.s[i + 1] * o.d[i + 1];
        double size = 1;
        for (int64_t x : o.d) size *= (double)x;
        if (size > 2147483647.0) fail(JET_EINVAL, "tensor larger than 2^31 elements");
    };
    load(A, rank_a, labels_a, dims_a);
    load(B, rank_b, labels_b, dims_b);
    auto pos = [](const std::vector<int64_t> &v, int64_t x) {
        for (size_t i = 0; i < v.size(); ++i)
            if (v[i] == x) return (int)i;
        return -1;
    };
    // output = A's free labels then B's free labels; summed = shared labels
    std::vector<int64_t> out, od, oa, ob, K, kd, ka, kb;
    for (size_t i = 0; i < A.l.size(); ++i) {
        int p = pos(B.l, A.l[i]);
        if (p < 0) {
            out.push_back(A.l[i]);
            od.push_back(A.d[i]);
            oa.push_back(A.s[i]);
            ob.push_back(0);
        } else {
            if (B.d[p] != A.d[i]) fail(JET_EINVAL, "shared label with different dims");
            K.push_back(A.l[i]);
            kd.push_back(A.d[i]);
            ka.push_back(A.s[i]);
            kb.push_back(B.s[p]);
        }
    }
    for (size_t i = 0; i < B.l.size(); ++i)
        if (pos(A.l, B.l[i]) < 0) {
            out.push_back(B.l[i]);
            od.push_back(B.d[i]);
            oa.push_back(0);
            ob.push_back(B.s[i]);
        }
    int64_t n_out = 1;
    for (int64_t x : od) n_out *= x;
    if (n_out > NOALLOC_MAX_OUT)
        fail(JET_EINVAL, "output has " + std::to_string(n_out) + " elements; the allocation-free contraction supports at most " +
                             std::to_string(NOALLOC_MAX_OUT));

    DirectArgs d;
    std::memset(&d, 0, sizeof d);
    // output split: cols = longest suffix with <= JET_COLMAX entries, rows decoded by loop
    size_t nc = 0;
    int64_t ncols = 1;
    while (nc < out.size() && ncols * od[out.size() - 1 - nc] <= JET_COLMAX) ncols *= od[out.size() - 1 - nc++];
    std::vector<int32_t> colA(ncols), colB(ncols);
    for (int64_t c = 0; c < ncols; ++c) {
        int64_t r = c, x = 0, y = 0;
        for (size_t j = 0; j < nc; ++j) {
            size_t li = out.size() - 1 - j;
            x += (r % od[li]) * oa[li];
            y += (r % od[li]) * ob[li];
            r /= od[li];
        }
        colA[c] = (int32_t)x;
        colB[c] = (int32_t)y;
    }
    d.n_cols = (int32_t)ncols;
    d.row_rank = (int32_t)(out.size() - nc);
    d.n_rows = 1;
    for (int j = 0; j < d.row_rank; ++j) {
        size_t li = out.size() - nc - 1 - j;
        d.row_dim[j] = od[li];
        d.row_sA[j] = oa[li];
        d.row_sB[j] = ob[li];
        d.n_rows *= od[li];
    }
    // summed index: klo = longest suffix (A's order) with <= JET_KLOMAX entries
    size_t nk = 0;
    int64_t nklo = 1;
    while (nk < K.size() && nklo * kd[K.size() - 1 - nk] <= JET_KLOMAX) nklo *= kd[K.size() - 1 - nk++];
    std::vector<int32_t> tkA(nklo), tkB(nklo);
    for (int64_t q = 0; q < nklo; ++q) {
        int64_t r = q, x = 0, y = 0;
        for (size_t j = 0; j < nk; ++j) {
            size_t li = K.size() - 1 - j;
            x += (r % kd[li]) * ka[li];
            y += (r % kd[li]) * kb[li];
            r /= kd[li];
        }
        tkA[q] = (int32_t)x;
        tkB[q] = (int32_t)y;
    }
    d.n_klo = (int32_t)nklo;
    d.khi_rank = (int32_t)(K.size() - nk);
    d.n_khi = 1;
    for (int j = 0; j < d.khi_rank; ++j) {
        size_t li = K.size() - nk - 1 - j;
        d.khi_dim[j] = kd[li];
        d.khi_sA[j] = ka[li];
        d.khi_sB[j] = kb[li];
        d.n_khi *= kd[li];
    }
    d.n_out = n_out;
    d.n_inst = 1;
    // split the summed index over as many blocks as the partials area holds
    const int64_t cap_partials = (int64_t)((NOALLOC_SCRATCH_BYTES - NOALLOC_TABLE_BYTES) / sizeof(float2));
    const int64_t groups = (n_out + JET_SPLITK_G - 1) / JET_SPLITK_G;
    int64_t parts = std::max<int64_t>(1, (148 * 8 + groups - 1) / groups);
    parts = std::min<int64_t>(parts, d.n_khi);
    parts = std::min<int64_t>(parts, cap_partials / n_out);
    d.khi_per_part = (int32_t)((d.n_khi + parts - 1) / parts);
    d.ksplit = (int32_t)((d.n_khi + d.khi_per_part - 1) / d.khi_per_part);

    // stage the tables and address slots into the scratch, then launch on the caller's stream
    int prev = -1;
    check(cudaGetDevice(&prev), "cudaGetDevice");
    check(cudaSetDevice(device), "cudaSetDevice");
    struct Restore {
        int dev;
        ~Restore() { cudaSetDevice(dev); }
    } restore{prev};
    unsigned char *scratch = (unsigned char *)noalloc_scratch_address(device);
    std::vector<unsigned char> host(NOALLOC_TABLE_BYTES, 0);
    size_t off = 0;
    auto put = [&](const void *src, size_t n) {
        size_t at = off;
        std::memcpy(host.data() + at, src, n);
        off = (off + n + 15) / 16 * 16;
        return at;
    };
    uint64_t pa = (uint64_t)a_dev, pb = (uint64_t)b_dev, pc = (uint64_t)c_dev;
    size_t o_pa = put(&pa, 8), o_pb = put(&pb, 8), o_pc = put(&pc, 8);
    size_t o_ca = put(colA.data(), colA.size() * 4), o_cb = put(colB.data(), colB.size() * 4);
    size_t o_ka = put(tkA.data(), tkA.size() * 4), o_kb = put(tkB.data(), tkB.size() * 4);
    cudaStream_t s = (cudaStream_t)stream;
    check(cudaMemcpyAsync(scratch, host.data(), off, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(tables)");
    d.ptrA = (uint64_t)(scratch + o_pa);
    d.ptrB = (uint64_t)(scratch + o_pb);
    d.ptrC = (uint64_t)(scratch + o_pc);
    d.colA = (uint64_t)(scratch + o_ca);
    d.colB = (uint64_t)(scratch + o_cb);
    d.kA = (uint64_t)(scratch + o_ka);
    d.kB = (uint64_t)(scratch + o_kb);
    d.partials = (uint64_t)(scratch + NOALLOC_TABLE_BYTES);   // every partial is written before it is read

    bool pow2 = true;
    for (int j = 0; j < d.row_rank; ++j) pow2 = pow2 && (d.row_dim[j] & (d.row_dim[j] - 1)) == 0;
    for (int j = 0; j < d.khi_rank; ++j) pow2 = pow2 && (d.khi_dim[j] & (d.khi_dim[j] - 1)) == 0;
    LaunchCfg c{d.ksplit, (int)groups, 1, 256, (int)(8 * nklo), 2 | (pow2 ? 4 : 0)};
    cudaGetLastError();
    check(launch_direct(d, c, s), "split-K contraction launch");
    SplitKReduceArgs r;
    std::memset(&r, 0, sizeof r);
    r.partials = d.partials;
    r.ptrC = d.ptrC;
    r.n_out = n_out;
    r.n_inst = 1;
    r.ksplit = d.ksplit;
    LaunchCfg rc{(int)std::min<int64_t>((n_out + 255) / 256, 65535), 1, 1, 256, 0, 0};
    check(launch_splitk_reduce(r, rc, s), "split-K reduction launch");
}

}  // namespace jet
