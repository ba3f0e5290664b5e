// rtproj_sketch_noalloc: the float64 sketch S = A G for callers that cannot allocate.
//
// Every other entry point of this library takes its scratch from a workspace the caller
// allocates. Some callers cannot do that: applications whose device memory is entirely
// owned by a pooling allocator or a fixed budget (a cudaMalloc would fail or fragment the
// pool), and latency-critical loops that must not pay cudaMalloc's implicit device
// synchronization. This entry point needs no workspace: the split-K partial sums of the
// sketch live in one fixed array of this library, g_sketch_scratch, 32 MiB in device
// memory (4 Mi float64 entries), which every GPU that loads the library holds until the
// process exits. The caller still passes A and the output S.
//
// Set-up: the first call on each device looks up the device address of the array with
// cudaGetSymbolAddress, with that device current; make that first call before any
// stream capture. All calls share the array and it keeps the last call's contents (each
// call overwrites every slab entry it reads, so nothing needs clearing); calls that
// overlap on the GPU race on it, so serialize them (one stream, or events).
#include "rtproj_internal.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr int64_t kScratchDoubles = 4ll << 20;   // 32 MiB
constexpr int NB_M = 64, NB_N = 64, NB_K = 16, NB_T = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_sketch_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Partial slab z of S = A G over the K range of split z (G entries from Philox, as in
// rtproj_sketch). Tile 64 x 64, 4 x 4 outputs per thread, float64 FMAs.
__global__ void __launch_bounds__(NB_T) sketch_partial_kernel(const double* A, int64_t lda, int m, int n, int l,
                                                              uint32_t key0, uint32_t key1, int dist, int kps,
                                                              double* part) {
    __shared__ double As[NB_K][NB_M + 1];
    __shared__ double Gs[NB_K][NB_N + 1];
    const int i0 = blockIdx.y * NB_M, j0 = blockIdx.x * NB_N, z = blockIdx.z;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int kbeg = z * kps, kend = min(n, kbeg + kps);
    double acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += NB_K) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = t + NB_T * r;
            const int ii = e / NB_K, kk = e % NB_K;
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < m && gk < kend) ? A[(int64_t)gi * lda + gk] : 0.0;
        }
        if (t < NB_N) {
            const int gj = j0 + t;
            uint4 w = make_uint4(0, 0, 0, 0);
            if (gj < l) w = rtp::philox4x32_10(make_uint4((uint32_t)(k0 >> 4), (uint32_t)gj, 0u, 0u), key0, key1);
#pragma unroll
            for (int kk = 0; kk < NB_K; ++kk)
                Gs[kk][t] = (gj < l && k0 + kk < kend) ? (double)rtp::omega_from_byte(rtp::block_byte(w, kk), dist) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < NB_K; ++kk) {
            double a[4], g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty * 4 + q]; g[q] = Gs[kk][tx * 4 + q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], g[y], acc[x][y]);
        }
        __syncthreads();
    }
    double* slab = part + (int64_t)z * m * l;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int gi = i0 + ty * 4 + x;
        if (gi >= m) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gj = j0 + tx * 4 + y;
            if (gj < l) slab[(int64_t)gi * l + gj] = acc[x][y];
        }
    }
}

__global__ void sketch_reduce_kernel(const double* part, int splits, int m, int l, double* S, int64_t lds) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)m * l;
    if (idx >= total) return;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * total + idx];
    S[(idx / l) * lds + idx % l] = s;
}

// Device address of g_sketch_scratch on the current device (looked up once per device).
rtproj_status scratch_on_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RTPROJ_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sketch_scratch) != cudaSuccess || !p) return RTPROJ_ECUDA;
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return RTPROJ_OK;
}

}  // namespace

extern "C" rtproj_status rtproj_sketch_noalloc(const double* A, int64_t m, int64_t n, int64_t lda, uint64_t seed,
                                               int64_t l, int omega, double* S, int64_t lds, void* stream) {
    if (!A || !S || m < 1 || n < m || lda < n || l < m || l > n || lds < l) return RTPROJ_EINVAL;
    if (omega != RTPROJ_OMEGA_UNIFORM && omega != RTPROJ_OMEGA_RADEMACHER) return RTPROJ_EINVAL;
    if (n > (int64_t)1 << 30) return RTPROJ_EUNSUPPORTED;
    const int64_t slab = m * l;
    if (slab > kScratchDoubles) return RTPROJ_ENOMEM;    // one partial slab must fit the fixed array
    // the array's address is per device: the stream must run on the current device
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return RTPROJ_ECUDA;
    if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) return RTPROJ_EINVAL;
    if (sdev != cur) return RTPROJ_EINVAL;
    double* part = nullptr;
    const rtproj_status st = scratch_on_current_device(&part);
    if (st != RTPROJ_OK) return st;
    const int tiles_m = (int)((m + NB_M - 1) / NB_M), tiles_n = (int)((l + NB_N - 1) / NB_N);
    const int tiles = tiles_m * tiles_n;
    int64_t splits = std::max<int64_t>(1, (4 * (int64_t)rtp::sm_count() + tiles - 1) / tiles);
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, (n + 255) / 256));
    splits = std::min<int64_t>(splits, kScratchDoubles / slab);
    int64_t kps = (n + splits - 1) / splits;
    kps = (kps + NB_K - 1) / NB_K * NB_K;
    splits = (n + kps - 1) / kps;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid(tiles_n, tiles_m, (unsigned)splits);
    sketch_partial_kernel<<<grid, NB_T, 0, s>>>(A, lda, (int)m, (int)n, (int)l, (uint32_t)(seed & 0xFFFFFFFFull),
                                                (uint32_t)(seed >> 32), omega, (int)kps, part);
    rtp::note_launch();
    sketch_reduce_kernel<<<(unsigned)((slab + 255) / 256), 256, 0, s>>>(part, (int)splits, (int)m, (int)l, S, lds);
    rtp::note_launch();
    return cudaGetLastError() == cudaSuccess ? RTPROJ_OK : RTPROJ_ECUDA;
}
