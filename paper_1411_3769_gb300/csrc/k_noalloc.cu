// Allocation-free variant of the tensor-core GEMM entry point.
//
// Some callers cannot call cudaMalloc at the point where they need the
// product: allocator or memory-pool callbacks (allocating there re-enters the
// allocator), and hosts that hand the library a fixed device budget up front
// and account for every byte.  This entry point takes device pointers for its
// inputs and its output.  Its scratch is the 16-byte-padded, TF32-split copy of
// A and B that the TMA loads read.  That scratch lives in one file-scope device
// array below, which every GPU that loads the library holds until the process
// exits.  The call is synchronous: it reads the kernel's timeout flag back and
// waits for its stream before it returns.
#include "psdp_internal.h"

// Largest (M + N) * Kpad the scratch holds, Kpad = K rounded up to 64:
// 2^20 floats (4 MiB) per copy; the hi and lo copies plus the flag word make
// 8 MiB + 256 B of device memory per GPU.
#define PSDP_NOALLOC_FLOATS (1 << 20)

static __device__ __align__(256) float g_noalloc_scratch[2 * PSDP_NOALLOC_FLOATS + 64];

namespace {

// Device address of the scratch array on the current device, looked up on every
// call (a host-side table lookup), so a context that was reset and re-created
// never sees a stale address.  The host-side name of the array is only a
// stand-in and must never be passed to a kernel.  Also sets the GEMM kernels'
// shared-memory limit on the current device.
psdp_status noalloc_scratch(float** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PSDP_ECUDA;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PSDP_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return PSDP_ECUDA;
    if (set_attrs_tc_gemm_fp32(optin) != cudaSuccess) return PSDP_ECUDA;
    *out = static_cast<float*>(p);
    return PSDP_OK;
}

// dst rows of length kpad from src rows of length k (zero padding); with lo
// non-null the value is split into TF32 hi + FP32 remainder lo.
__global__ void k_pack_rows(const float* __restrict__ src, int rows, int k, int kpad, float* hi, float* lo) {
    const int64_t total = (int64_t)rows * kpad;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / kpad;
        const int c = (int)(i % kpad);
        const float v = (c < k) ? src[r * k + c] : 0.f;
        if (lo) {
            uint32_t h;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
            hi[i] = __uint_as_float(h);
            lo[i] = v - __uint_as_float(h);
        } else {
            hi[i] = v;
        }
    }
}

void pack(cudaStream_t st, const float* src, int rows, int k, int kpad, float* hi, float* lo) {
    int64_t blocks = ((int64_t)rows * kpad + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_pack_rows<<<(int)blocks, 256, 0, st>>>(src, rows, k, kpad, hi, lo);
}

}  // namespace

// Same product as psdp_tc_gemm_check (dtype 0), on device buffers and without
// allocating: C[n*M + m] = sum_k A[m*K + k] * B[n*K + k].  Synchronous on
// `stream`.  Calls that overlap on the GPU share the scratch and race.  A CUDA
// error that earlier work left unread is reported as ECUDA before anything is
// enqueued and is left for its owner to read; a failure of this call's own
// runtime calls or launches gives ECUDA too.
extern "C" psdp_status psdp_tc_gemm_noalloc(int M, int N, int K, int split, const float* A, const float* B, float* C,
                                            void* stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || (split != 1 && split != 3)) return PSDP_EINVAL;
    const int64_t kpad = ((int64_t)K + 63) / 64 * 64;
    if (((int64_t)M + N) * kpad > PSDP_NOALLOC_FLOATS) return PSDP_EINVAL;
    if (cudaPeekAtLastError() != cudaSuccess) return PSDP_ECUDA;
    float* base = nullptr;
    const psdp_status s0 = noalloc_scratch(&base);
    if (s0 != PSDP_OK) return s0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* hiA = base;
    float* hiB = base + (int64_t)M * kpad;
    float* loA = base + PSDP_NOALLOC_FLOATS;
    float* loB = loA + (int64_t)M * kpad;
    int* flag = reinterpret_cast<int*>(base + 2 * PSDP_NOALLOC_FLOATS);
    // the scratch keeps the previous call's contents: the timeout flag starts at zero
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return PSDP_ECUDA;
    CUtensorMap mA, mB, mAl, mBl;
    bool ok = tc_make_map(&mA, hiA, false, K, M, 1, kpad, 0, 128) && tc_make_map(&mB, hiB, false, K, N, 1, kpad, 0, 128);
    if (ok && split == 3)
        ok = tc_make_map(&mAl, loA, false, K, M, 1, kpad, 0, 128) && tc_make_map(&mBl, loB, false, K, N, 1, kpad, 0, 128);
    if (!ok) return PSDP_ECUDA;
    pack(st, A, M, K, (int)kpad, hiA, split == 3 ? loA : nullptr);
    pack(st, B, N, K, (int)kpad, hiB, split == 3 ? loB : nullptr);
    launch_tc_gemm(st, false, split, mA, mB, split == 3 ? &mAl : nullptr, split == 3 ? &mBl : nullptr, M, N, 1, 0,
                   nullptr, K, C, M, 0, 1.f, 0.f, 0, flag);
    if (cudaGetLastError() != cudaSuccess) return PSDP_ECUDA;   // the three launches above
    int h_flag = 0;
    if (cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PSDP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PSDP_ECUDA;
    return h_flag ? PSDP_ETIMEOUT : PSDP_OK;
}
