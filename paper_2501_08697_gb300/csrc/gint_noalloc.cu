// gint_block_dot_noalloc: the block-store inner product <A, B> without any allocation.
//
// Why: some callers cannot call cudaMalloc (or anything that may allocate) at the point
// where they need the result: code running inside a custom allocator or a memory-pool
// callback, code that must not change device-memory usage once a steady state has been
// reached, or hosts that forbid allocation after start-up.  gint_block_dot keeps its
// partial sums in scratch owned by the handle; this variant keeps them in a fixed
// file-scope device array instead, so the call itself allocates nothing.
//
// The array is a static __device__ symbol: every GPU that loads the library holds
// kNoAllocPartials doubles (8 KiB) until the process exits.  Its address is looked up on
// every call (cudaGetSymbolAddress in the current context, which allocates nothing), so no
// address outlives the context it belongs to.  All calls share the array, so calls that
// overlap on the GPU (e.g. on two streams) race and give wrong sums.  Each call overwrites
// the partials it uses, so nothing needs clearing between calls.
#include "gint_internal.h"

namespace {

constexpr int kNoAllocPartials = 1024;               // partial sums held by the static array
constexpr int kNoAllocChunk = 65536;                 // values reduced by one block
constexpr int kNoAllocThreads = 256;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

// block b sums A[i] * B[i] over its contiguous chunk [b * kNoAllocChunk, ...) in a fixed order
__global__ void k_dot_chunks(const double *__restrict__ A, const double *__restrict__ B, int64_t n, double *part)
{
    __shared__ double sh[kNoAllocThreads];
    const int64_t lo = (int64_t)blockIdx.x * kNoAllocChunk;
    const int64_t hi = lo + kNoAllocChunk < n ? lo + kNoAllocChunk : n;
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += A[i] * B[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dot_sum(const double *part, int nblk, double *out)
{
    __shared__ double sh[kNoAllocThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

}  // namespace

extern "C" gint_status gint_block_dot_noalloc(gint_handle h, const double *A_dev, const double *B_dev,
                                              double *out_dev, void *stream)
{
    gint_status st = gint::check_handle(h, "gint_block_dot_noalloc");
    if (st != GINT_OK) return st;
    if (!A_dev || !B_dev || !out_dev) {
        gint::set_error("gint_block_dot_noalloc: null argument");
        return GINT_EINVAL;
    }
    const int64_t n = h->info.nvalues;
    if (n > (int64_t)kNoAllocPartials * kNoAllocChunk) {
        gint::set_error("gint_block_dot_noalloc: %lld values exceed the static scratch limit of %lld "
                        "(%d partial sums of %d values); use gint_block_dot",
                        (long long)n, (long long)kNoAllocPartials * kNoAllocChunk, kNoAllocPartials, kNoAllocChunk);
        return GINT_EINVAL;
    }
    // the symbol's address in the current context (host code cannot use the symbol's name as a
    // device pointer)
    void *part_v = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&part_v, g_noalloc_partials);
    if (e != cudaSuccess) return gint::cuda_fail(e, "gint_block_dot_noalloc: cudaGetSymbolAddress");
    double *part = (double *)part_v;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = n > 0 ? (int)((n + kNoAllocChunk - 1) / kNoAllocChunk) : 0;
    if (nblk > 0) k_dot_chunks<<<nblk, kNoAllocThreads, 0, s>>>(A_dev, B_dev, n, part);
    k_dot_sum<<<1, kNoAllocThreads, 0, s>>>(part, nblk, out_dev);
    e = cudaGetLastError();
    return e == cudaSuccess ? GINT_OK : gint::cuda_fail(e, "gint_block_dot_noalloc: launch");
}
