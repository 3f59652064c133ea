// Auxiliary kernels: the CPML tensor admission rule (Sec. 2.3), the bounding box of the pole
// mask, a NaN/Inf scan, and the BF16 snapshot codec with one scale per slab (Sec. 3.2).
#include <cuda_bf16.h>

#include "fdtd_internal.cuh"

namespace gbfdtd {

// Sec. 2.3: inside an absorbing face a tensor is admitted only if the face normal is a principal
// axis with a non-intermediate eigenvalue.  For a diagonal tensor the normal of a q-face is a
// principal axis; reject a cell of a q-slab whose eps_qq lies strictly between the other two
// (the same order test on 1/eps).
template <typename T>
__global__ void k_admission(const Dom<T>* __restrict__ dd, unsigned long long* bad) {
    const Dom<T>& d = *dd;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= d.ncell) return;
    const int i = (int)(t % d.n[0]);
    const int j = (int)((t / d.n[0]) % d.n[1]);
    const int k = (int)(t / ((long long)d.n[0] * d.n[1]));
    const int c[3] = {i, j, k};
    const T v[3] = {d.ie[0][t], d.ie[1][t], d.ie[2][t]};
    for (int q = 0; q < 3; ++q) {
        if (d.ns[q] == 0 || slab_of(c[q], d.dlo[q], d.dhi[q], d.n[q]) < 0) continue;
        const T a = v[(q + 1) % 3], b = v[(q + 2) % 3], x = v[q];
        const T lo = a < b ? a : b, hi = a < b ? b : a;
        if (x > lo && x < hi) {
            atomicAdd(bad, 1ull);
            return;
        }
    }
}

__global__ void k_mask_box(const uint8_t* __restrict__ mask, int nx, int ny, int nz, int* box) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nx * ny * nz) return;
    if (!mask[t]) return;
    const int i = (int)(t % nx), j = (int)((t / nx) % ny), k = (int)(t / ((long long)nx * ny));
    atomicMin(box + 0, i);
    atomicMin(box + 1, j);
    atomicMin(box + 2, k);
    atomicMax(box + 3, i + 1);
    atomicMax(box + 4, j + 1);
    atomicMax(box + 5, k + 1);
}

template <typename T>
__global__ void k_nonfinite(const T* __restrict__ p, long long n, unsigned long long* bad) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const T v = p[t];
        if (!(v == v) || v - v != T(0)) {  // NaN fails v == v; +-Inf gives Inf - Inf = NaN
            atomicAdd(bad, 1ull);
            return;
        }
    }
}

// BF16 snapshot codec, one FP32 scale per slab (outermost index): s = max |x| over the slab,
// q = bf16_rn(x / s), x' = float(q) * s.  Grids are (blocks per slab, slabs): many blocks per slab
// and no index division.  The scale is reduced with an atomic max on the float's bits (valid for
// non-negative values; NaN is ignored by fmaxf, as in a sequential max).
template <typename T>
__global__ void __launch_bounds__(256) k_slab_absmax(const T* __restrict__ src, long long plane,
                                                     unsigned* __restrict__ scale_bits) {
    const long long base = (long long)blockIdx.y * plane;
    float m = 0.f;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < plane; t += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf((float)src[base + t]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        atomicMax(scale_bits + blockIdx.y, __float_as_uint(m));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_bf16_quant(const T* __restrict__ src, long long plane,
                                                    const float* __restrict__ scales, __nv_bfloat16* __restrict__ dst) {
    // divide (not multiply by 1/s): a slab whose max is an FP32 denormal has 1/s = inf, and
    // 0 * inf would store NaN; x / s stays within [-1, 1]
    const float s = scales[blockIdx.y];
    const long long base = (long long)blockIdx.y * plane;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < plane; t += (long long)gridDim.x * blockDim.x)
        dst[base + t] = __float2bfloat16_rn(s > 0.f ? (float)src[base + t] / s : 0.f);
}

template <typename T>
__global__ void __launch_bounds__(256) k_bf16_decode(const __nv_bfloat16* __restrict__ src,
                                                     const float* __restrict__ scales, long long plane,
                                                     T* __restrict__ dst) {
    const float s = scales[blockIdx.y];
    const long long base = (long long)blockIdx.y * plane;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < plane; t += (long long)gridDim.x * blockDim.x)
        dst[base + t] = (T)(__bfloat162float(src[base + t]) * s);
}

// blocks per slab: about 8 elements per thread, at most 64 blocks
inline unsigned codec_blocks(long long plane) {
    const long long b = (plane + 256 * 8 - 1) / (256 * 8);
    return (unsigned)(b < 1 ? 1 : (b > 64 ? 64 : b));
}

// Net Poynting flux along +z through the H plane of a two-plane monitor (Sec. 2.4), one block
// per frequency: P = 1/2 Re sum [ (Ex(k) + Ex(k+1))/2 conj(Hy(k)) - (Ey(k) + Ey(k+1))/2 conj(Hx(k)) ]
// over the monitor's x-y cells.  sEx..sHy: accumulator slots of the four components.
__global__ void __launch_bounds__(256) k_flux(const Mon* __restrict__ mon, int sEx, int sEy, int sHx, int sHy,
                                              double* __restrict__ out) {
    const Mon& m = *mon;
    const int f = blockIdx.x;
    const long long plane = (long long)m.bx * m.by;
    const double2* ex = m.acc + ((long long)sEx * m.nf + f) * m.ncell;
    const double2* ey = m.acc + ((long long)sEy * m.nf + f) * m.ncell;
    const double2* hx = m.acc + ((long long)sHx * m.nf + f) * m.ncell;
    const double2* hy = m.acc + ((long long)sHy * m.nf + f) * m.ncell;
    double sum = 0.0;
    for (long long c = threadIdx.x; c < plane; c += blockDim.x) {
        const double2 a0 = ex[c], a1 = ex[c + plane], b0 = ey[c], b1 = ey[c + plane];
        const double2 gx = hx[c], gy = hy[c];
        const double exr = 0.5 * (a0.x + a1.x), exi = 0.5 * (a0.y + a1.y);
        const double eyr = 0.5 * (b0.x + b1.x), eyi = 0.5 * (b0.y + b1.y);
        // Re(E conj(H)) = Er Hr + Ei Hi
        sum += 0.5 * ((exr * gy.x + exi * gy.y) - (eyr * gx.x + eyi * gx.y));
    }
    __shared__ double red[256];
    red[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = red[0];
}

void launch_flux(const Launch& L, const Mon* mon, int nf, const int* slots, double* out) {
    if (nf <= 0) return;
    k_flux<<<nf, 256, 0, L.stream>>>(mon, slots[0], slots[1], slots[2], slots[3], out);
    ++*L.counter;
}

template <typename T>
void launch_admission(const Launch& L, const Dom<T>* d_dom, const Dom<T>& h_dom, unsigned long long* d_bad) {
    const int bs = 256;
    k_admission<T><<<(unsigned)((h_dom.ncell + bs - 1) / bs), bs, 0, L.stream>>>(d_dom, d_bad);
    ++*L.counter;
}

void launch_mask_box(const Launch& L, const uint8_t* mask, int nx, int ny, int nz, int* d_box) {
    const int bs = 256;
    const long long n = (long long)nx * ny * nz;
    k_mask_box<<<(unsigned)((n + bs - 1) / bs), bs, 0, L.stream>>>(mask, nx, ny, nz, d_box);
    ++*L.counter;
}

template <typename T>
void launch_nonfinite(const Launch& L, const T* p, long long n, unsigned long long* d_bad) {
    if (n <= 0) return;
    const int bs = 256;
    long long blocks = (n + bs - 1) / bs;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_nonfinite<T><<<(unsigned)blocks, bs, 0, L.stream>>>(p, n, d_bad);
    ++*L.counter;
}

template <typename T>
void launch_bf16_encode(const Launch& L, const T* src, long long nplanes, long long plane, uint16_t* dst,
                        float* scales) {
    if (nplanes <= 0 || plane <= 0) return;
    const dim3 g(codec_blocks(plane), (unsigned)nplanes);
    cudaMemsetAsync(scales, 0, sizeof(float) * nplanes, L.stream);
    k_slab_absmax<T><<<g, 256, 0, L.stream>>>(src, plane, reinterpret_cast<unsigned*>(scales));
    k_bf16_quant<T><<<g, 256, 0, L.stream>>>(src, plane, scales, reinterpret_cast<__nv_bfloat16*>(dst));
    *L.counter += 2;
}

template <typename T>
void launch_bf16_decode(const Launch& L, const uint16_t* src, const float* scales, long long nplanes,
                        long long plane, T* dst) {
    if (nplanes <= 0 || plane <= 0) return;
    const dim3 g(codec_blocks(plane), (unsigned)nplanes);
    k_bf16_decode<T><<<g, 256, 0, L.stream>>>(reinterpret_cast<const __nv_bfloat16*>(src), scales, plane, dst);
    ++*L.counter;
}

// ---- native snapshots ----------------------------------------------------------------------
// One launch moves every state part between the live arrays and a snapshot slot: block row y
// copies segment y, grid-stride along x.  Slot offsets are 256-byte aligned; a part array starts
// on a 256-byte boundary (fields, CPML memories) or at least on its element size (pole-state parts
// inside one allocation), and its size is a whole number of elements of >= 4 bytes.  16-byte
// vectors where both ends are 16-byte aligned (the last bytes % 16 bytes by lanes of block x = 0),
// 4-byte words otherwise.
__global__ void k_snapshot_copy(const SnapSeg* __restrict__ segs, char* __restrict__ slot, int to_slot) {
    const SnapSeg sg = segs[blockIdx.y];
    const char* src = to_slot ? sg.state : slot + sg.off;
    char* dst = to_slot ? slot + sg.off : sg.state;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, dt = (long long)gridDim.x * blockDim.x;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
        const long long nv = sg.bytes >> 4;
        const int4* s4 = reinterpret_cast<const int4*>(src);
        int4* d4 = reinterpret_cast<int4*>(dst);
        for (long long v = t0; v < nv; v += dt) d4[v] = s4[v];
        const int tail = (int)(sg.bytes & 15);
        if (blockIdx.x == 0 && (int)threadIdx.x < tail) dst[(nv << 4) + threadIdx.x] = src[(nv << 4) + threadIdx.x];
    } else {
        const long long nw = sg.bytes >> 2;
        const unsigned* s1 = reinterpret_cast<const unsigned*>(src);
        unsigned* d1 = reinterpret_cast<unsigned*>(dst);
        for (long long v = t0; v < nw; v += dt) d1[v] = s1[v];
    }
}

void launch_snapshot_copy(const Launch& L, const SnapSeg* segs, int nseg, long long max_bytes, void* slot,
                          int to_slot) {
    if (nseg <= 0) return;
    long long bx = ((max_bytes >> 4) + 256 * 8 - 1) / (256 * 8);   // <= 8 vectors per thread
    bx = bx < 1 ? 1 : (bx > 1024 ? 1024 : bx);
    k_snapshot_copy<<<dim3((unsigned)bx, (unsigned)nseg), 256, 0, L.stream>>>(segs, (char*)slot, to_slot);
    ++*L.counter;
}

#define GBFDTD_INST(T)                                                                                     \
    template void launch_admission<T>(const Launch&, const Dom<T>*, const Dom<T>&, unsigned long long*);   \
    template void launch_nonfinite<T>(const Launch&, const T*, long long, unsigned long long*);             \
    template void launch_bf16_encode<T>(const Launch&, const T*, long long, long long, uint16_t*, float*); \
    template void launch_bf16_decode<T>(const Launch&, const uint16_t*, const float*, long long, long long, T*);
GBFDTD_INST(float)
GBFDTD_INST(double)
#undef GBFDTD_INST

}  // namespace gbfdtd
