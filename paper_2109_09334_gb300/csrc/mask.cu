// mask.cu -- crowded-flavor masking (Sec. 3.1): the pixels affected by
// saturated sources, for the mask argument of the build.
//
// A pixel is masked (0) when R or S reaches its saturation level anywhere in
// the square of half-width `grow` around it (Chebyshev distance, clipped at
// the image edges) or when the input mask masks it; else kept (1).
// One block per 32 x 32 output tile: the saturation flags of the tile and
// its halo are staged in shared memory, then dilated along y and along x.
#include <cuda_runtime.h>

#include "internal.h"

namespace sfft {

constexpr int kMaskTile = 32;
constexpr int kMaxGrow = 16;

template <typename I>
__global__ void __launch_bounds__(256) k_sat_mask(int n0, int n1, const I *__restrict__ R, const I *__restrict__ S,
                                                  double sat_r, double sat_s, int grow,
                                                  const uint8_t *mask_in, uint8_t *mask_out) {
    constexpr int E = kMaskTile + 2 * kMaxGrow;
    __shared__ uint8_t flag[E][E];        // [x][y] of tile + halo
    __shared__ uint8_t hdil[E][kMaskTile];  // dilated along y
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int x0 = blockIdx.y * kMaskTile, y0 = blockIdx.x * kMaskTile;
    const int ext = kMaskTile + 2 * grow;
    for (int i = ty; i < ext; i += 8)
        for (int j = tx; j < ext; j += 32) {
            const int x = x0 - grow + i, y = y0 - grow + j;
            uint8_t f = 0;
            if (x >= 0 && x < n0 && y >= 0 && y < n1) {
                const size_t k = (size_t)x * n1 + y;
                f = ((double)R[k] >= sat_r || (double)S[k] >= sat_s) ? 1 : 0;
            }
            flag[i][j] = f;
        }
    __syncthreads();
    for (int i = ty; i < ext; i += 8) {
        uint8_t h = 0;
        for (int d = 0; d <= 2 * grow; ++d) h |= flag[i][tx + d];
        hdil[i][tx] = h;
    }
    __syncthreads();
    for (int i = ty; i < kMaskTile; i += 8) {
        const int x = x0 + i, y = y0 + tx;
        if (x >= n0 || y >= n1) continue;
        uint8_t v = 0;
        for (int d = 0; d <= 2 * grow; ++d) v |= hdil[i + d][tx];
        const size_t k = (size_t)x * n1 + y;
        const uint8_t keep = (v == 0 && (mask_in == nullptr || mask_in[k] != 0)) ? 1 : 0;
        mask_out[k] = keep;
    }
}

}  // namespace sfft

using namespace sfft;

extern "C" int sfft_saturation_mask(int32_t n0, int32_t n1, int32_t dtype, const void *d_ref, const void *d_sci,
                                    double sat_ref, double sat_sci, int32_t grow, const uint8_t *d_mask_in,
                                    uint8_t *d_mask_out, sfft_stream_t stream) {
    if (!d_ref || !d_sci || !d_mask_out) return SFFT_ERR_INVALID;
    if (n0 < 1 || n1 < 1 || grow < 0 || grow > kMaxGrow) return SFFT_ERR_INVALID;
    if (dtype != SFFT_F32 && dtype != SFFT_F64) return SFFT_ERR_INVALID;
    dim3 grid((n1 + kMaskTile - 1) / kMaskTile, (n0 + kMaskTile - 1) / kMaskTile);
    dim3 block(32, 8);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SFFT_F32)
        k_sat_mask<float><<<grid, block, 0, s>>>(n0, n1, (const float *)d_ref, (const float *)d_sci, sat_ref,
                                                 sat_sci, grow, d_mask_in, d_mask_out);
    else
        k_sat_mask<double><<<grid, block, 0, s>>>(n0, n1, (const double *)d_ref, (const double *)d_sci, sat_ref,
                                                  sat_sci, grow, d_mask_in, d_mask_out);
    return status_of(cudaGetLastError());
}
