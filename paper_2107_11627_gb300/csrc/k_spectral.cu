// Wavelength-dependent colour (Sec. 3.5): one channel of n NHWC frames copied
// to or from single-channel planes, so that each colour channel can run the
// whole path on its own context (its wavelength's basis and network scaling).
#include "p2s_internal.h"

namespace p2s {

namespace {

struct ChanPtrs {
    const float *src[kMaxBatch];
    float *dst[kMaxBatch];
};

// dst[f][p * dst_stride + dst_off] = src[f][p * src_stride + src_off] for the npx pixels of
// frame f = blockIdx.y
__global__ void __launch_bounds__(256) channel_copy_kernel(ChanPtrs ptr, long long npx, int src_stride, int src_off,
                                                           int dst_stride, int dst_off) {
    const float *s = ptr.src[blockIdx.y];
    float *d = ptr.dst[blockIdx.y];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx; p += (long long)gridDim.x * blockDim.x)
        d[p * dst_stride + dst_off] = __ldg(s + p * src_stride + src_off);
}

}  // namespace

p2s_status launch_channel_copy(const float *const *src, float *const *dst, int n, long long npx, int src_stride,
                               int src_off, int dst_stride, int dst_off, cudaStream_t st) {
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int nb = n - i0 < kMaxBatch ? n - i0 : kMaxBatch;
        ChanPtrs p;
        for (int i = 0; i < nb; ++i) {
            p.src[i] = src[i0 + i];
            p.dst[i] = dst[i0 + i];
        }
        const long long want = (npx + 255) / 256;
        dim3 grid((unsigned)(want < 4096 ? want : 4096), nb);
        if (npx > 0) channel_copy_kernel<<<grid, 256, 0, st>>>(p, npx, src_stride, src_off, dst_stride, dst_off);
        P2S_CUDA(cudaGetLastError());
    }
    return P2S_OK;
}

}  // namespace p2s
