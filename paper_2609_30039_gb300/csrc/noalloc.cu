// Allocation-free variant of the non-finite scan (see fdtd_count_nonfinite_noalloc in
// include/fdtd.h).  The method of the paper has no counterpart: this entry point serves callers
// that must not allocate device memory.
//
// Scratch: one file-scope __device__ array of kNoallocPartials per-block counts plus one total.
// Every process that loads the library holds it on every GPU it touches until exit.  Host code
// must not pass the symbol itself to a kernel (on the host it is only a stand-in): its device
// address is looked up with cudaGetSymbolAddress, with the caller's device current, on every
// call.  The lookup costs little next to the synchronisation each call ends with, and an address
// kept from an earlier call could point at released memory once the device's context has been
// torn down and recreated (cudaDeviceReset), when the array may have moved.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fdtd.h"

namespace {

constexpr int kNoallocPartials = 2048;   // per-block partial counts held in the scratch array
constexpr int kNoallocThreads = 256;
constexpr long long kNoallocPerThread = 64;
constexpr long long kNoallocMaxValues = (long long)kNoallocPartials * kNoallocThreads * kNoallocPerThread;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoallocPartials + 1];

template <typename T>
__global__ void k_count_nonfinite_partial(const T* __restrict__ p, long long n, unsigned long long* partial) {
    unsigned long long cnt = 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const T v = p[t];
        cnt += (!(v == v) || v - v != T(0)) ? 1ull : 0ull;
    }
    __shared__ unsigned long long red[kNoallocThreads / 32];
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kNoallocThreads / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;   // every slot below gridDim.x is rewritten by each call
    }
}

__global__ void k_count_nonfinite_total(unsigned long long* partial, int nblocks) {
    unsigned long long s = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ unsigned long long red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partial[kNoallocPartials] = t;
    }
}

}  // namespace

extern "C" fdtd_status fdtd_count_nonfinite_noalloc(const void* data, int64_t n, int32_t dtype, void* stream,
                                                     int64_t* count) {
    if (!count || n < 0 || (n > 0 && !data) || (dtype != FDTD_F32 && dtype != FDTD_F64)) return FDTD_EINVAL;
    if (n > kNoallocMaxValues) return FDTD_EINVAL;   // needs more than kNoallocPartials partial counts
    *count = 0;
    if (n == 0) return FDTD_OK;
    // the scratch array's address on the current device (see the file comment)
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FDTD_ECUDA;
    unsigned long long* scratch = (unsigned long long*)p;
    const cudaStream_t st = (cudaStream_t)stream;
    long long blocks = (n + kNoallocThreads * kNoallocPerThread - 1) / (kNoallocThreads * kNoallocPerThread);
    if (blocks < 1) blocks = 1;
    if (dtype == FDTD_F32)
        k_count_nonfinite_partial<float><<<(unsigned)blocks, kNoallocThreads, 0, st>>>((const float*)data, n, scratch);
    else
        k_count_nonfinite_partial<double><<<(unsigned)blocks, kNoallocThreads, 0, st>>>((const double*)data, n, scratch);
    k_count_nonfinite_total<<<1, 1024, 0, st>>>(scratch, (int)blocks);
    if (cudaGetLastError() != cudaSuccess) return FDTD_ECUDA;
    unsigned long long total = 0;
    if (cudaMemcpyAsync(&total, scratch + kNoallocPartials, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FDTD_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FDTD_ECUDA;
    *count = (int64_t)total;
    return FDTD_OK;
}
