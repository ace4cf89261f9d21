// Device scans and a stable LSD radix sort of (uint64 key, int32 value) pairs,
// used to order the elements along the Morton curve that defines the octree
// (Sec. 3.3 Step 1: the octree is built as in FMM / kernel-independent FMM).
#include "fda_internal.cuh"

namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

// block-wide exclusive scan of one value per thread; returns the block total
template <typename T>
__device__ T block_exclusive_scan(T v, T *sh, T &total)
{
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int off = 1; off < blockDim.x; off <<= 1) {
        T a = (t >= off) ? sh[t - off] : T(0);
        __syncthreads();
        sh[t] += a;
        __syncthreads();
    }
    total = sh[blockDim.x - 1];
    T incl = sh[t];
    __syncthreads();
    return incl - v;
}

template <typename T>
__global__ void k_tile_sums(const T *in, int64_t n, T *sums)
{
    __shared__ T sh[SCAN_T];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
    for (int r = 0; r < SCAN_ITEMS; ++r)
        if (base + r < n) s += in[base + r];
    T tot;
    block_exclusive_scan<T>(s, sh, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// exclusive scan of a short array by one block (sequential chunks per thread)
template <typename T>
__global__ void k_scan_small(T *a, int64_t n, T *total_out)
{
    __shared__ T sh[1024];
    int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
    int64_t b = (int64_t)threadIdx.x * chunk, e = b + chunk < n ? b + chunk : n;
    T s = 0;
    for (int64_t i = b; i < e; ++i) s += a[i];
    T tot;
    T off = block_exclusive_scan<T>(s, sh, tot);
    for (int64_t i = b; i < e; ++i) {
        T v = a[i];
        a[i] = off;
        off += v;
    }
    if (threadIdx.x == 0 && total_out) *total_out = tot;
}

template <typename T>
__global__ void k_tile_scan(const T *in, T *out, int64_t n, const T *tile_off)
{
    __shared__ T sh[SCAN_T];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
    for (int r = 0; r < SCAN_ITEMS; ++r)
        if (base + r < n) s += in[base + r];
    T tot;
    T off = block_exclusive_scan<T>(s, sh, tot) + tile_off[blockIdx.x];
    for (int r = 0; r < SCAN_ITEMS; ++r)
        if (base + r < n) {
            T v = in[base + r];
            out[base + r] = off;
            off += v;
        }
}

template <typename T>
void exclusive_scan(const T *in, T *out, int64_t n, cudaStream_t s, T *total_host)
{
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return;
    }
    int64_t ntile = (n + SCAN_TILE - 1) / SCAN_TILE;
    T *sums = nullptr, *tot = nullptr;
    FDA_CUDA(cudaMallocAsync((void **)&sums, sizeof(T) * (ntile + 1), s));
    tot = sums + ntile;
    k_tile_sums<T><<<(unsigned)ntile, SCAN_T, 0, s>>>(in, n, sums);
    FDA_CHECK_LAUNCH();
    k_scan_small<T><<<1, 1024, 0, s>>>(sums, ntile, tot);
    FDA_CHECK_LAUNCH();
    k_tile_scan<T><<<(unsigned)ntile, SCAN_T, 0, s>>>(in, out, n, sums);
    FDA_CHECK_LAUNCH();
    if (total_host) {
        FDA_CUDA(cudaMemcpyAsync(total_host, tot, sizeof(T), cudaMemcpyDeviceToHost, s));
        FDA_CUDA(cudaStreamSynchronize(s));
    }
    FDA_CUDA(cudaFreeAsync(sums, s));
}

// ---------------------------------------------------------------------------
// radix sort: 8-bit digits, tiles of 256 threads x 16 items, stable
// ---------------------------------------------------------------------------
constexpr int RS_T = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_T * RS_ITEMS;

__global__ void k_rs_hist(const uint64_t *keys, int64_t n, int shift, int32_t *hist, int ntile)
{
    __shared__ int32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntile + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout, int64_t n,
                             int shift, const int32_t *hist, int ntile)
{
    __shared__ int32_t base_d[256];
    __shared__ int32_t run[256];
    __shared__ int32_t wcnt[RS_T / 32][257];
    int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    base_d[t] = hist[(int64_t)t * ntile + blockIdx.x];
    run[t] = 0;
    unsigned lt_mask = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        for (int w = 0; w < RS_T / 32; ++w) wcnt[w][t] = 0;
        if (t == 0)
            for (int w = 0; w < RS_T / 32; ++w) wcnt[w][256] = 0;
        __syncthreads();
        int64_t i = base + r * RS_T + t;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int lrank = __popc(peers & lt_mask);
        int leader = __ffs(peers) - 1;
        if (lane == leader) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = base_d[d] + run[d] + lrank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
        int add = 0;
        for (int w = 0; w < RS_T / 32; ++w) add += wcnt[w][t];
        run[t] += add;
        __syncthreads();
    }
}

}  // namespace

void fda_exclusive_scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s, int32_t *total_host)
{
    exclusive_scan<int32_t>(in, out, n, s, total_host);
}

void fda_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s, int64_t *total_host)
{
    exclusive_scan<int64_t>(in, out, n, s, total_host);
}

void fda_radix_sort_u64(uint64_t *keys, int32_t *vals, int64_t n, int key_bits, cudaStream_t s)
{
    if (n <= 1) return;
    int ntile = (int)((n + RS_TILE - 1) / RS_TILE);
    uint64_t *k2 = nullptr;
    int32_t *v2 = nullptr, *hist = nullptr;
    FDA_CUDA(cudaMallocAsync((void **)&k2, sizeof(uint64_t) * n, s));
    FDA_CUDA(cudaMallocAsync((void **)&v2, sizeof(int32_t) * n, s));
    FDA_CUDA(cudaMallocAsync((void **)&hist, sizeof(int32_t) * 256 * (int64_t)ntile, s));
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int passes = (key_bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_hist<<<ntile, RS_T, 0, s>>>(ka, n, shift, hist, ntile);
        FDA_CHECK_LAUNCH();
        exclusive_scan<int32_t>(hist, hist, (int64_t)256 * ntile, s, nullptr);
        k_rs_scatter<<<ntile, RS_T, 0, s>>>(ka, va, kb, vb, n, shift, hist, ntile);
        FDA_CHECK_LAUNCH();
        uint64_t *tk = ka; ka = kb; kb = tk;
        int32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        FDA_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        FDA_CUDA(cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    FDA_CUDA(cudaFreeAsync(k2, s));
    FDA_CUDA(cudaFreeAsync(v2, s));
    FDA_CUDA(cudaFreeAsync(hist, s));
}
