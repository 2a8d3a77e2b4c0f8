// codec.cu -- 8-bit log depth codec (ImLoc Sec. 3.3 "Data Compression":
// depth clipped to [0.25 m, 128 m], quantized in log space with 256 levels;
// Sec. 4.3 "Depth Quantization": under 1.4 % relative error).
//
// Code 0 = no depth; code c in 1..255 stands for 0.25 * 512^((c-1)/254) m.
// The encoder decides each code by exact comparisons with the 254 level
// midpoints (each held as the smallest float32 not below the FP64 midpoint,
// so that d >= T holds exactly when d lies at or above the midpoint), not by
// a rounded logarithm: codes do not depend on a transcendental function's
// last bits.  The decode table (code -> float32 metres, FP64 values rounded
// to nearest) is the one the lift kernel reads its taps through.
//
// Also the two blocked float32 layouts of the map store that the lift
// addresses: 4x4-pixel blocks (imloc_depth_tile4_async) and overlapping
// 8x4-pixel blocks every 7 x 3 pixels (imloc_depth_halo_async).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "codec.h"
#include "common.cuh"

namespace imloc {

namespace {

struct CodecTables {
    float mid[kLog8Levels - 1];  // smallest float >= midpoint between codes c and c+1 (c = 1..254)
    float dec[256];              // code -> metres (code 0 -> 0)
};

const CodecTables& tables() {
    static CodecTables T;
    static std::once_flag once;
    std::call_once(once, [] {
        for (int c = 1; c < kLog8Levels; ++c) {
            const double m = 0.25 * pow(512.0, (c - 0.5) / 254.0);
            float f = static_cast<float>(m);
            if (static_cast<double>(f) < m) f = nextafterf(f, INFINITY);
            T.mid[c - 1] = f;
        }
        T.dec[0] = 0.0f;
        for (int c = 1; c < 256; ++c) T.dec[c] = static_cast<float>(0.25 * pow(512.0, (c - 1) / 254.0));
    });
    return T;
}

struct EncodeParams {
    const float* depth;
    uint8_t* codes;
    int64_t pitch, code_pitch;
    int32_t W, H;
    float mid[kLog8Levels - 1];
};

struct DecodeParams {
    const uint8_t* codes;
    float* out;
    int64_t code_pitch, out_pitch;
    int32_t W, H;
    float dec[256];
};

constexpr int kCodecThreads = 256;

__global__ void __launch_bounds__(kCodecThreads) k_depth_encode(const __grid_constant__ EncodeParams p) {
    __shared__ float s_mid[256];
    for (int i = threadIdx.x; i < 256; i += kCodecThreads) s_mid[i] = i < kLog8Levels - 1 ? p.mid[i] : INFINITY;
    __syncthreads();
    const int64_t n = static_cast<int64_t>(p.W) * p.H;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * kCodecThreads + threadIdx.x; k < n;
         k += static_cast<int64_t>(gridDim.x) * kCodecThreads) {
        const int y = static_cast<int>(k / p.W), x = static_cast<int>(k - static_cast<int64_t>(y) * p.W);
        const float d = __ldg(p.depth + static_cast<int64_t>(y) * p.pitch + x);
        uint8_t code = 0;
        if (d > 0.0f && d < INFINITY) {
            // number of midpoints at or below d (binary search over the 254 ascending midpoints;
            // the padding entries are +inf)
            int lo = 0;
#pragma unroll
            for (int step = 128; step >= 1; step >>= 1)
                if (d >= s_mid[lo + step - 1]) lo += step;
            code = static_cast<uint8_t>(1 + lo);
        }
        p.codes[static_cast<int64_t>(y) * p.code_pitch + x] = code;
    }
}

__global__ void __launch_bounds__(kCodecThreads) k_depth_decode(const __grid_constant__ DecodeParams p) {
    __shared__ float s_dec[256];
    for (int i = threadIdx.x; i < 256; i += kCodecThreads) s_dec[i] = p.dec[i];
    __syncthreads();
    const int64_t n = static_cast<int64_t>(p.W) * p.H;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * kCodecThreads + threadIdx.x; k < n;
         k += static_cast<int64_t>(gridDim.x) * kCodecThreads) {
        const int y = static_cast<int>(k / p.W), x = static_cast<int>(k - static_cast<int64_t>(y) * p.W);
        p.out[static_cast<int64_t>(y) * p.out_pitch + x] = s_dec[__ldg(p.codes + static_cast<int64_t>(y) * p.code_pitch + x)];
    }
}

int grid_for(int64_t n) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 132;
    const int64_t want = (n + kCodecThreads - 1) / kCodecThreads;
    return static_cast<int>(want < 8LL * sms ? (want > 0 ? want : 1) : 8LL * sms);
}

}  // namespace

void log8_decode_table(float out[256]) { memcpy(out, tables().dec, sizeof(float) * 256); }

}  // namespace imloc

extern "C" {

int imloc_depth_encode_log8_async(const float* depth, int32_t width, int32_t height, int64_t pitch,
                                  uint8_t* codes, int64_t code_pitch, void* stream) {
    using namespace imloc;
    if (!depth || !codes || width < 1 || height < 1 || pitch < width || code_pitch < width) return IMLOC_ERR_INVALID_ARG;
    EncodeParams p;
    p.depth = depth;
    p.codes = codes;
    p.pitch = pitch;
    p.code_pitch = code_pitch;
    p.W = width;
    p.H = height;
    memcpy(p.mid, tables().mid, sizeof(p.mid));
    const int64_t n = static_cast<int64_t>(width) * height;
    k_depth_encode<<<grid_for(n), kCodecThreads, 0, static_cast<cudaStream_t>(stream)>>>(p);
    IMLOC_CUDA_TRY(cudaGetLastError());
    return IMLOC_OK;
}

int imloc_depth_decode_log8_async(const uint8_t* codes, int32_t width, int32_t height, int64_t code_pitch,
                                  float* out, int64_t out_pitch, void* stream) {
    using namespace imloc;
    if (!codes || !out || width < 1 || height < 1 || code_pitch < width || out_pitch < width) return IMLOC_ERR_INVALID_ARG;
    DecodeParams p;
    p.codes = codes;
    p.out = out;
    p.code_pitch = code_pitch;
    p.out_pitch = out_pitch;
    p.W = width;
    p.H = height;
    memcpy(p.dec, tables().dec, sizeof(p.dec));
    const int64_t n = static_cast<int64_t>(width) * height;
    k_depth_decode<<<grid_for(n), kCodecThreads, 0, static_cast<cudaStream_t>(stream)>>>(p);
    IMLOC_CUDA_TRY(cudaGetLastError());
    return IMLOC_OK;
}

}  // extern "C"

// ---- blocked float32 layout (4x4 pixels per 64-byte block) -----------------
namespace imloc {
namespace {
// one thread per output element: consecutive threads write consecutive
// elements of a block row; each group of 4 reads 4 consecutive pixels
__global__ void __launch_bounds__(256) k_depth_tile4(const float* __restrict__ depth, int64_t pitch, int32_t W,
                                                     int32_t H, float* __restrict__ tiled, int64_t tiled_pitch,
                                                     int64_t total) {
    for (int64_t o = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x; o < total;
         o += static_cast<int64_t>(gridDim.x) * 256) {
        const int64_t by = o / tiled_pitch, r = o - by * tiled_pitch;
        const int64_t bx = r >> 4, k = r & 15;
        const int64_t y = 4 * by + (k >> 2), x = 4 * bx + (k & 3);
        tiled[o] = (x < W && y < H) ? __ldg(depth + y * pitch + x) : 0.0f;
    }
}
}  // namespace
}  // namespace imloc

extern "C" int imloc_depth_tile4_async(const float* depth, int32_t width, int32_t height, int64_t pitch, float* tiled,
                                       int64_t tiled_pitch, void* stream) {
    if (!depth || !tiled || width < 1 || height < 1 || pitch < width) return IMLOC_ERR_INVALID_ARG;
    if (tiled_pitch % 16 != 0 || tiled_pitch < 16 * ((static_cast<int64_t>(width) + 3) / 4)) return IMLOC_ERR_INVALID_ARG;
    const int64_t total = ((static_cast<int64_t>(height) + 3) / 4) * tiled_pitch;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    imloc::k_depth_tile4<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        depth, pitch, width, height, tiled, tiled_pitch, total);
    IMLOC_CUDA_TRY(cudaGetLastError());
    return IMLOC_OK;
}

// ---- overlapping-block float32 layout (8x4-pixel blocks every 7 x 3 pixels) --
namespace imloc {
namespace {
// one thread per output element: consecutive threads write consecutive
// elements of a block row; each group of 8 reads 8 consecutive pixels
__global__ void __launch_bounds__(256) k_depth_halo(const float* __restrict__ depth, int64_t pitch, int32_t W,
                                                    int32_t H, float* __restrict__ halo, int64_t halo_pitch,
                                                    int64_t total) {
    for (int64_t o = static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x; o < total;
         o += static_cast<int64_t>(gridDim.x) * 256) {
        const int64_t by = o / halo_pitch, r = o - by * halo_pitch;
        const int64_t bx = r >> 5, k = r & 31;
        const int64_t y = 3 * by + (k >> 3), x = 7 * bx + (k & 7);
        halo[o] = (x < W && y < H) ? __ldg(depth + y * pitch + x) : 0.0f;
    }
}
}  // namespace
}  // namespace imloc

extern "C" int imloc_depth_halo_async(const float* depth, int32_t width, int32_t height, int64_t pitch, float* halo,
                                      int64_t halo_pitch, void* stream) {
    if (!depth || !halo || width < 1 || height < 1 || pitch < width) return IMLOC_ERR_INVALID_ARG;
    if (halo_pitch % 32 != 0 || halo_pitch < 32 * ((static_cast<int64_t>(width) - 1) / 7 + 1))
        return IMLOC_ERR_INVALID_ARG;
    const int64_t total = ((static_cast<int64_t>(height) - 1) / 3 + 1) * halo_pitch;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
    imloc::k_depth_halo<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        depth, pitch, width, height, halo, halo_pitch, total);
    IMLOC_CUDA_TRY(cudaGetLastError());
    return IMLOC_OK;
}
