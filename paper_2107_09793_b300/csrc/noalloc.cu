// Allocation-free pairwise contraction (jet_pair_contract_noalloc).
//
// For callers that must not allocate device memory: a serving process whose
// GPU memory is pre-reserved by its own allocator (a cudaMalloc behind its back
// can fail or fragment that pool), or a latency-critical loop where cudaMalloc /
// cudaFree would add implicit device synchronisation.  The caller passes device
// inputs and a device output; the split-K partial sums and the offset tables
// live in one fixed, file-scope device array instead of the plan workspace.
#include <cuda_runtime.h>

#include <algorithm>
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

// The offset tables and the three address slots, written into the scratch by
// one small kernel from the labels' dims and strides (passed by value), so that
// no host staging buffer or host-to-device copy is involved.
constexpr int NOALLOC_TABLE_LABELS = 16;   // a 1024-entry table spans at most 10 labels of dim >= 2
struct NoallocTableArgs {
    uint64_t slots;                        // 3 uint64 address slots (A, B, C)
    uint64_t pa, pb, pc;
    uint64_t colA, colB, kA, kB;           // int32 tables
    int32_t ncols, nklo, nc, nk;
    int64_t cdim[NOALLOC_TABLE_LABELS], csA[NOALLOC_TABLE_LABELS], csB[NOALLOC_TABLE_LABELS];   // fastest first
    int64_t kdim[NOALLOC_TABLE_LABELS], ksA[NOALLOC_TABLE_LABELS], ksB[NOALLOC_TABLE_LABELS];
};

__global__ void noalloc_tables_kernel(NoallocTableArgs t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        uint64_t *slot = (uint64_t *)t.slots;
        slot[0] = t.pa;
        slot[1] = t.pb;
        slot[2] = t.pc;
    }
    if (i < t.ncols) {
        int64_t r = i, x = 0, y = 0;
        for (int j = 0; j < t.nc; ++j) {
            const int64_t v = r % t.cdim[j];
            x += v * t.csA[j];
            y += v * t.csB[j];
            r /= t.cdim[j];
        }
        ((int32_t *)t.colA)[i] = (int32_t)x;
        ((int32_t *)t.colB)[i] = (int32_t)y;
    }
    if (i < t.nklo) {
        int64_t r = i, x = 0, y = 0;
        for (int j = 0; j < t.nk; ++j) {
            const int64_t v = r % t.kdim[j];
            x += v * t.ksA[j];
            y += v * t.ksB[j];
            r /= t.kdim[j];
        }
        ((int32_t *)t.kA)[i] = (int32_t)x;
        ((int32_t *)t.kB)[i] = (int32_t)y;
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
    // A label of dim 1 has the single value 0: it moves no offset and is left
    // out of the output and summed decodes (the output's row-major layout is
    // the same with or without it).
    for (size_t i = 0; i < A.l.size(); ++i) {
        int p = pos(B.l, A.l[i]);
        if (p >= 0 && B.d[p] != A.d[i]) fail(JET_EINVAL, "shared label with different dims");
        if (A.d[i] == 1) continue;
        if (p < 0) {
            out.push_back(A.l[i]);
            od.push_back(A.d[i]);
            oa.push_back(A.s[i]);
            ob.push_back(0);
        } else {
            K.push_back(A.l[i]);
            kd.push_back(A.d[i]);
            ka.push_back(A.s[i]);
            kb.push_back(B.s[p]);
        }
    }
    for (size_t i = 0; i < B.l.size(); ++i)
        if (B.d[i] > 1 && pos(A.l, B.l[i]) < 0) {
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
    if (out.size() - nc > (size_t)JET_MAXR)
        fail(JET_EINVAL, "output rank too large (at most " + std::to_string(JET_MAXR) + " labels of dim > 1 besides "
                         "the fastest " + std::to_string(nc) + ")");
    NoallocTableArgs t;
    std::memset(&t, 0, sizeof t);
    t.nc = (int32_t)nc;
    for (size_t j = 0; j < nc; ++j) {
        size_t li = out.size() - 1 - j;
        t.cdim[j] = od[li];
        t.csA[j] = oa[li];
        t.csB[j] = ob[li];
    }
    t.ncols = (int32_t)ncols;
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
    if (K.size() - nk > (size_t)JET_MAXR)
        fail(JET_EINVAL, "too many summed labels (at most " + std::to_string(JET_MAXR) + " of dim > 1 besides "
                         "the fastest " + std::to_string(nk) + ")");
    t.nk = (int32_t)nk;
    for (size_t j = 0; j < nk; ++j) {
        size_t li = K.size() - 1 - j;
        t.kdim[j] = kd[li];
        t.ksA[j] = ka[li];
        t.ksB[j] = kb[li];
    }
    t.nklo = (int32_t)nklo;
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

    // write the tables and address slots into the scratch, then launch on the caller's stream
    int prev = -1;
    check(cudaGetDevice(&prev), "cudaGetDevice");
    check(cudaSetDevice(device), "cudaSetDevice");
    struct Restore {
        int dev;
        ~Restore() { cudaSetDevice(dev); }
    } restore{prev};
    // an error left pending by the caller's earlier CUDA work is reported, not cleared
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        fail(JET_ECUDA, std::string("a CUDA error was pending before the call: ") + cudaGetErrorString(pending));
    unsigned char *scratch = (unsigned char *)noalloc_scratch_address(device);
    size_t off = 0;
    auto place = [&](size_t n) {
        size_t at = off;
        off = (off + n + 15) / 16 * 16;
        return at;
    };
    const size_t o_slots = place(3 * 8);
    const size_t o_ca = place((size_t)ncols * 4), o_cb = place((size_t)ncols * 4);
    const size_t o_ka = place((size_t)nklo * 4), o_kb = place((size_t)nklo * 4);
    if (off > NOALLOC_TABLE_BYTES) fail(JET_EINVAL, "offset tables exceed the scratch table area");
    t.slots = (uint64_t)(scratch + o_slots);
    t.pa = (uint64_t)a_dev;
    t.pb = (uint64_t)b_dev;
    t.pc = (uint64_t)c_dev;
    t.colA = (uint64_t)(scratch + o_ca);
    t.colB = (uint64_t)(scratch + o_cb);
    t.kA = (uint64_t)(scratch + o_ka);
    t.kB = (uint64_t)(scratch + o_kb);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_tab = std::max<int64_t>({ncols, nklo, 1});
    noalloc_tables_kernel<<<(unsigned)((n_tab + 255) / 256), 256, 0, s>>>(t);
    check(cudaGetLastError(), "offset-table launch");
    d.ptrA = t.slots;
    d.ptrB = t.slots + 8;
    d.ptrC = t.slots + 16;
    d.colA = t.colA;
    d.colB = t.colB;
    d.kA = t.kA;
    d.kB = t.kB;
    d.partials = (uint64_t)(scratch + NOALLOC_TABLE_BYTES);   // every partial is written before it is read

    bool pow2 = true;
    for (int j = 0; j < d.row_rank; ++j) pow2 = pow2 && (d.row_dim[j] & (d.row_dim[j] - 1)) == 0;
    for (int j = 0; j < d.khi_rank; ++j) pow2 = pow2 && (d.khi_dim[j] & (d.khi_dim[j] - 1)) == 0;
    LaunchCfg c{d.ksplit, (int)groups, 1, 256, (int)(8 * nklo), 2 | (pow2 ? 4 : 0)};
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
