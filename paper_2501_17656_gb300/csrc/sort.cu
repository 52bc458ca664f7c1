// sort.cu -- device-wide exclusive scan and stable LSD radix sort (8-bit digits).
#include "internal.h"

namespace h2mg {

struct TempBuf {
  void* p = nullptr;
  explicit TempBuf(size_t bytes) {
    if (bytes) H2_CUDA(cudaMalloc(&p, bytes));
  }
  ~TempBuf() {
    if (p) best_effort(cudaFree(p), "cudaFree (sort scratch)");
  }
  template <class T>
  T* as() { return static_cast<T*>(p); }
};

// ----------------------------------------------------------------------------- scan
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ int block_exclusive_scan(int v, int* sh, int& total) {
  // sh: SCAN_THREADS/32 ints
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < SCAN_THREADS / 32 ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < SCAN_THREADS / 32) sh[lane] = s;
  }
  __syncthreads();
  total = sh[SCAN_THREADS / 32 - 1];
  int excl = x - v + (w > 0 ? sh[w - 1] : 0);
  __syncthreads();
  return excl;
}

__global__ void k_scan_reduce(const int* __restrict__ in, int n, int* __restrict__ sums) {
  __shared__ int sh[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int acc = 0;
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
    if (i < n) acc += in[i];
  }
  int total;
  block_exclusive_scan(acc, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_single(int* __restrict__ v, int n) {
  // exclusive scan of n values by one block, in chunks of SCAN_THREADS
  __shared__ int sh[SCAN_THREADS / 32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += SCAN_THREADS) {
    int i = base + threadIdx.x;
    int x = i < n ? v[i] : 0;
    int total;
    int e = block_exclusive_scan(x, sh, total);
    int c = carry;
    if (i < n) v[i] = e + c;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const int* __restrict__ in, int n, const int* __restrict__ sums,
                             int* __restrict__ out) {
  __shared__ int sh[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int loc[SCAN_ITEMS];
  int acc = 0;
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    loc[j] = acc;
    if (i < n) acc += in[i];
  }
  int total;
  int e = block_exclusive_scan(acc, sh, total);
  int off = sums[blockIdx.x] + e;
  for (int j = 0; j < SCAN_ITEMS; ++j) {
    int64_t i = base + j;
    if (i < n) out[i] = off + loc[j];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = sums[blockIdx.x] + total;
}

// out[0..n] = exclusive scan of in[0..n-1]; out[n] = total. `in` and `out` may alias.
void exclusive_scan_i32(const int* in, int* out, int n, cudaStream_t s, Matrix&) {
  if (n <= 0) {
    H2_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
    return;
  }
  int nb = ceil_div(n, SCAN_TILE);
  TempBuf sums(sizeof(int) * (nb + 1));
  TempBuf tmp(sizeof(int) * (size_t)n);
  H2_CUDA(cudaMemcpyAsync(tmp.p, in, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  { k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(tmp.as<int>(), n, sums.as<int>()); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  { k_scan_single<<<1, SCAN_THREADS, 0, s>>>(sums.as<int>(), nb); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  { k_scan_apply<<<nb, SCAN_THREADS, 0, s>>>(tmp.as<int>(), n, sums.as<int>(), out); ::h2mg::count_launch(); }
  H2_LAUNCH_CHECK();
  H2_CUDA(cudaStreamSynchronize(s));   // temporaries are freed on return
}

// ----------------------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;                          // items per thread
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;       // 2048 items per tile
constexpr int RS_WARP_ITEMS = 32 * RS_ROUNDS;         // contiguous items of one warp

__device__ __forceinline__ int rs_index(int tile, int w, int r, int lane) {
  return tile * RS_TILE + w * RS_WARP_ITEMS + r * 32 + lane;
}

__global__ void k_rs_hist(const uint64_t* __restrict__ key, int n, int shift, int ntiles,
                          int* __restrict__ hist) {
  __shared__ int h[256];
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) h[d] = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int i = rs_index(blockIdx.x, w, r, lane);
    if (i < n) atomicAdd(&h[(int)((key[i] >> shift) & 255u)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) hist[d * ntiles + blockIdx.x] = h[d];
}

__global__ void k_rs_scatter(const uint64_t* __restrict__ key, const int* __restrict__ val,
                             uint64_t* __restrict__ key_out, int* __restrict__ val_out, int n,
                             int shift, int ntiles, const int* __restrict__ offs) {
  __shared__ int wcount[RS_THREADS / 32][257];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = lane; d < 257; d += 32) wcount[w][d] = 0;
  __syncwarp();
  int dig[RS_ROUNDS], rank[RS_ROUNDS];
  uint64_t kk[RS_ROUNDS];
  int vv[RS_ROUNDS];
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int i = rs_index(blockIdx.x, w, r, lane);
    int d = 256;
    if (i < n) {
      kk[r] = key[i];
      vv[r] = val[i];
      d = (int)((kk[r] >> shift) & 255u);
    }
    dig[r] = d;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int base = wcount[w][d];
    __syncwarp();
    int leader = __ffs(peers) - 1;
    if (lane == leader) wcount[w][d] = base + __popc(peers);
    __syncwarp();
    rank[r] = base + __popc(peers & lt);
  }
  __syncthreads();
  // exclusive prefix over warps for each digit
  for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
    int acc = 0;
    for (int ww = 0; ww < RS_THREADS / 32; ++ww) {
      int c = wcount[ww][d];
      wcount[ww][d] = acc;
      acc += c;
    }
  }
  __syncthreads();
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int d = dig[r];
    if (d < 256) {
      int pos = offs[d * ntiles + blockIdx.x] + wcount[w][d] + rank[r];
      key_out[pos] = kk[r];
      val_out[pos] = vv[r];
    }
  }
}

// Stable sort of (keys, vals) by the low `bits` bits of the keys (LSD, 8 bits per pass).
void radix_sort_u64(uint64_t* keys, int* vals, int n, int bits, Matrix& M, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  int ntiles = ceil_div(n, RS_TILE);
  TempBuf k2(sizeof(uint64_t) * (size_t)n), v2(sizeof(int) * (size_t)n);
  TempBuf hist(sizeof(int) * ((size_t)256 * ntiles + 1));
  uint64_t *ka = keys, *kb = k2.as<uint64_t>();
  int *va = vals, *vb = v2.as<int>();
  int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    { k_rs_hist<<<ntiles, RS_THREADS, 0, s>>>(ka, n, 8 * p, ntiles, hist.as<int>()); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    exclusive_scan_i32(hist.as<int>(), hist.as<int>(), 256 * ntiles, s, M);
    { k_rs_scatter<<<ntiles, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, 8 * p, ntiles, hist.as<int>()); ::h2mg::count_launch(); }
    H2_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    H2_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    H2_CUDA(cudaMemcpyAsync(vals, va, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  }
  H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace h2mg
