// An allocation-free variant of the tensor-core product (qed_tc_gemm): the split-K
// partial sums and the error word live in file-scope device arrays instead of memory
// obtained from cudaMalloc, and a second kernel adds the partials into the caller's
// output.  For callers that must not allocate device memory (for example code running
// inside another framework's memory pool, or a process whose allocations are fixed up
// front): it calls no cudaMalloc, cudaFree or allocating library routine.
#include <mutex>
#include <string>

#include "gemm_tc.h"
#include "kernels.h"
#include "model.h"

namespace qed {

// 16 MiB of split-K partial sums: splits * M * N <= kStaticScratchFloats.
constexpr int64_t kStaticScratchFloats = (int64_t)4 << 20;

static __device__ __align__(256) float g_static_scratch[kStaticScratchFloats];
static __device__ __align__(256) uint32_t g_static_err[64];

namespace {

constexpr int kMaxDevices = 64;

struct StaticPtrs {
    bool ready = false;
    float *scratch = nullptr;
    uint32_t *err = nullptr;
};

StaticPtrs g_ptrs[kMaxDevices];
std::mutex g_ptrs_mutex;  // first calls on a device from several host threads

// out[i] = sum over s of part[s * MN + i], in a fixed order
__global__ void sum_partials_kernel(int64_t MN, int splits, const float *part, float *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MN) return;
    float acc = part[i];
    for (int s = 1; s < splits; ++s) acc += part[s * MN + i];
    out[i] = acc;
}

// Device addresses of the file-scope arrays, looked up once per device with that device
// current (host code may not use the array names as device addresses).
qed_status static_ptrs(StaticPtrs *&p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        set_error("qed_tc_gemm_static: no usable current device");
        return QED_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_ptrs_mutex);
    p = &g_ptrs[dev];
    if (p->ready) return QED_OK;
    float *scratch = nullptr;
    uint32_t *err = nullptr;
    cudaError_t e1 = cudaGetSymbolAddress((void **)&scratch, g_static_scratch);
    cudaError_t e2 = cudaGetSymbolAddress((void **)&err, g_static_err);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("qed_tc_gemm_static: cudaGetSymbolAddress failed: ") +
                  cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        return QED_ECUDA;
    }
    p->scratch = scratch;
    p->err = err;
    p->ready = true;
    return QED_OK;
}

}  // namespace

}  // namespace qed

extern "C" qed_status qed_tc_gemm_static(const void *a_planes, int32_t planes_a, const void *b_planes,
                                         int32_t planes_b, int32_t M, int32_t N, int32_t K, int32_t n_seg,
                                         const int32_t *seg_pairs, int32_t splits, float *out, qed_stream stream) {
    using namespace qed;
    if (!a_planes || !b_planes || !out || !seg_pairs || M <= 0 || N <= 0 || K <= 0 || splits <= 0 || n_seg <= 0 ||
        n_seg > kTcMaxSeg) {
        set_error("qed_tc_gemm_static: bad argument");
        return QED_EINVAL;
    }
    if ((int64_t)splits * M * N > kStaticScratchFloats) {
        set_error("qed_tc_gemm_static: splits * M * N exceeds the static scratch of " +
                  std::to_string(kStaticScratchFloats) + " floats");
        return QED_EINVAL;
    }
    StaticPtrs *sp = nullptr;
    qed_status st = static_ptrs(sp);
    if (st != QED_OK) return st;
    TcGemm g;
    int pairs[2 * kTcMaxSeg];
    for (int q = 0; q < 2 * n_seg; ++q) pairs[q] = seg_pairs[q];
    if (!tc_gemm_plan(g, a_planes, planes_a, b_planes, planes_b, M, N, K, n_seg, pairs, 1, splits))
        return QED_EINVAL;
    if (g.splits != splits) {
        set_error("qed_tc_gemm_static: splits must divide the n_seg*K/64 k-blocks into that many non-empty slices");
        return QED_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(sp->err, 0, sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        set_error("qed_tc_gemm_static: cudaMemsetAsync failed");
        return QED_ECUDA;
    }
    // the partial sums are only read if the product's own launch was accepted (otherwise the
    // scratch still holds the previous call's partials)
    cudaError_t le = tc_gemm_launch(g, sp->scratch, sp->err, s);
    if (le != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("qed_tc_gemm_static: tensor-core launch failed: ") + cudaGetErrorString(le));
        return QED_ECUDA;
    }
    const int64_t MN = (int64_t)M * N;
    sum_partials_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, s>>>(MN, splits, sp->scratch, out);
    count_launches(1);
    le = cudaGetLastError();
    if (le != cudaSuccess) {
        set_error(std::string("qed_tc_gemm_static: summation launch failed: ") + cudaGetErrorString(le));
        return QED_ECUDA;
    }
    uint32_t h = 0;
    cudaMemcpyAsync(&h, sp->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_error(std::string("qed_tc_gemm_static: ") + cudaGetErrorString(e));
        return QED_ECUDA;
    }
    if (h & kErrTimeout) {
        set_error("qed_tc_gemm_static: a bounded wait ran out");
        return QED_ETIMEOUT;
    }
    return QED_OK;
}
