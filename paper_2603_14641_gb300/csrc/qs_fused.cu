// Fused gate segments: many consecutive layers per tableau pass.
//
// Every generator row evolves independently under the update rules (Sec. 2.4,
// Eq. 4: the rules apply to each row index i), so the 64 rows held by one
// column word w can run through a whole segment of layers -- up to the next
// measurement -- without any other row. A block loads word slice w (X[q][w],
// Z[q][w] for all n qubits, 16 n bytes) into shared memory, applies every gate
// of every layer of the segment there (gates of one layer touch disjoint
// qubits, so threads of one layer never collide; a barrier separates layers),
// accumulates its sign contributions in registers and writes the slice back
// once. Global traffic per segment drops from (layers x touched columns) to one
// read and one write of the tableau plus the gate records. The paper launches
// one kernel per window (Sec. 4.1, Alg. 2); this is the fused alternative for
// tableaus whose slice fits in the 227 KB of shared memory of an SM
// (n up to 14,080 qubits with one word per block).
#include <algorithm>

#include "qs_internal.cuh"
#include "qs_rules.cuh"

namespace qs {

// grid.x = ceil(nwords / WPB); block owns words [WPB * blockIdx.x, +WPB) of every column.
// lptr: L + 1 gate offsets (absolute indices into packed). R >= the gates of
// any layer / blockDim.x: a thread issues the loads of all its gate records of
// a layer (and the next layer's end offset) before it applies any of them, so
// each layer costs one memory latency rather than one per gate.
template <bool SIGNS, int WPB, int R>
__global__ void __launch_bounds__(1024)
fused_segment_kernel(uint64_t *__restrict__ X, uint64_t *__restrict__ Z, uint64_t *__restrict__ S,
                     uint32_t n, uint32_t stride, uint32_t nwords,
                     const uint32_t *__restrict__ packed, const int64_t *__restrict__ lptr,
                     uint32_t L, uint32_t *__restrict__ err) {
  extern __shared__ uint64_t sm[];
  uint64_t *sx = sm, *sz = sm + (size_t)n * WPB;
  const uint32_t w0 = blockIdx.x * WPB;
  for (uint32_t q = threadIdx.x; q < n; q += blockDim.x) {
#pragma unroll
    for (int j = 0; j < WPB; ++j) {
      const bool in = w0 + j < nwords;
      sx[q * WPB + j] = in ? X[(size_t)q * stride + w0 + j] : 0ull;
      sz[q * WPB + j] = in ? Z[(size_t)q * stride + w0 + j] : 0ull;
    }
  }
  __syncthreads();
  uint64_t sacc[WPB];
#pragma unroll
  for (int j = 0; j < WPB; ++j) sacc[j] = 0;
  bool bad = false;
  const uint2 *rec2 = reinterpret_cast<const uint2 *>(packed);
  int64_t ga = L ? lptr[0] : 0, gb = L ? lptr[1] : 0;
  for (uint32_t l = 0; l < L; ++l) {
    const int64_t gn = (l + 2 <= L) ? __ldg(lptr + l + 2) : gb;  // next layer's end
    uint2 rec[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int64_t g = ga + threadIdx.x + (int64_t)i * blockDim.x;
      rec[i] = g < gb ? __ldg(rec2 + g) : make_uint2(0, 0);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
      if (ga + threadIdx.x + (int64_t)i * blockDim.x >= gb) break;
      const uint32_t w = rec[i].x, qb = rec[i].y;
      const uint32_t type = w >> 24, qa = w & 0xFFFFFFu;
      const bool two = type >= QS_CX && type <= QS_ISWAP;
      if (qa >= n || type >= QS_NUM_GATE_TYPES || (two && (qb >= n || qb == qa))) {
        bad = true;
        continue;
      }
#pragma unroll
      for (int j = 0; j < WPB; ++j) {
        uint64_t xa = sx[qa * WPB + j], za = sz[qa * WPB + j], xb = 0, zb = 0;
        if (two) { xb = sx[qb * WPB + j]; zb = sz[qb * WPB + j]; }
        rule<SIGNS>(type, xa, za, xb, zb, sacc[j]);
        sx[qa * WPB + j] = xa;
        sz[qa * WPB + j] = za;
        if (two) { sx[qb * WPB + j] = xb; sz[qb * WPB + j] = zb; }
      }
    }
    __syncthreads();
    ga = gb;
    gb = gn;
  }
  if (bad && blockIdx.x == 0) atomicOr(err, kErrBadGate);
  for (uint32_t q = threadIdx.x; q < n; q += blockDim.x) {
#pragma unroll
    for (int j = 0; j < WPB; ++j) {
      if (w0 + j < nwords) {
        X[(size_t)q * stride + w0 + j] = sx[q * WPB + j];
        Z[(size_t)q * stride + w0 + j] = sz[q * WPB + j];
      }
    }
  }
  if (SIGNS) {
    __shared__ uint64_t red[WPB][32];
#pragma unroll
    for (int j = 0; j < WPB; ++j) {
      uint64_t v = sacc[j];
      for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < WPB && w0 + threadIdx.x < nwords) {
      uint64_t v = 0;
      for (uint32_t wp = 0; wp < (blockDim.x + 31) / 32; ++wp) v ^= red[threadIdx.x][wp];
      S[w0 + threadIdx.x] ^= v;
    }
  }
}

constexpr size_t kFusedSmemMax = 220 * 1024;
constexpr uint32_t kFusedThreads = 1024;

int fused_words_per_block(uint32_t n, uint32_t nwords) {
  // widest slice that fits shared memory while keeping at least one block per SM
  if ((size_t)16 * n > kFusedSmemMax) return 0;
  for (int wpb : {4, 2})
    if ((size_t)16 * n * wpb <= kFusedSmemMax && (nwords + wpb - 1) / wpb >= 152) return wpb;
  return 1;
}

bool fused_fits(uint32_t n) { return (size_t)16 * n <= kFusedSmemMax; }

template <bool SIGNS, int WPB, int R>
static cudaError_t launch_fused_t(uint64_t *X, uint64_t *Z, uint64_t *S, uint32_t n, uint32_t stride,
                                  uint32_t nwords, const uint32_t *packed, const int64_t *lptr,
                                  uint32_t L, uint32_t *err, cudaStream_t s) {
  static std::atomic<uint64_t> attr_set{0};  // one bit per device ordinal
  cudaError_t ea = once_per_device(attr_set, []() {
    return cudaFuncSetAttribute(fused_segment_kernel<SIGNS, WPB, R>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax);
  });
  if (ea != cudaSuccess) return ea;
  const size_t smem = (size_t)16 * n * WPB;
  const uint32_t blocks = (nwords + WPB - 1) / WPB;
  fused_segment_kernel<SIGNS, WPB, R><<<blocks, kFusedThreads, smem, s>>>(X, Z, S, n, stride, nwords,
                                                                          packed, lptr, L, err);
  return cudaGetLastError();
}

template <bool SIGNS, int WPB>
static cudaError_t launch_fused_r(uint32_t max_gates, uint64_t *X, uint64_t *Z, uint64_t *S, uint32_t n,
                                  uint32_t stride, uint32_t nwords, const uint32_t *packed,
                                  const int64_t *lptr, uint32_t L, uint32_t *err, cudaStream_t s) {
  // a layer holds at most n gates and a WPB-word slice of 16 n WPB bytes fits
  // 220 KB, so R <= 16 for one word, 8 for two and 4 for four
  const uint32_t r = (max_gates + kFusedThreads - 1) / kFusedThreads;
  if (r <= 1) return launch_fused_t<SIGNS, WPB, 1>(X, Z, S, n, stride, nwords, packed, lptr, L, err, s);
  if (r <= 2) return launch_fused_t<SIGNS, WPB, 2>(X, Z, S, n, stride, nwords, packed, lptr, L, err, s);
  if (r <= 4) return launch_fused_t<SIGNS, WPB, 4>(X, Z, S, n, stride, nwords, packed, lptr, L, err, s);
  if constexpr (WPB <= 2)
    if (r <= 8) return launch_fused_t<SIGNS, WPB, 8>(X, Z, S, n, stride, nwords, packed, lptr, L, err, s);
  if constexpr (WPB == 1)
    if (r <= 16) return launch_fused_t<SIGNS, WPB, 16>(X, Z, S, n, stride, nwords, packed, lptr, L, err, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fused_segment(uint64_t *X, uint64_t *Z, uint64_t *S, uint32_t n, uint32_t stride,
                                 uint32_t nwords, const uint32_t *packed, const int64_t *lptr,
                                 uint32_t L, uint32_t max_gates, uint32_t *err, cudaStream_t s) {
  const int wpb = fused_words_per_block(n, nwords);
  const bool signs = S != nullptr;
#define QS_FUSED_CASE(W)                                                                          \
  if (wpb == W)                                                                                   \
    return signs ? launch_fused_r<true, W>(max_gates, X, Z, S, n, stride, nwords, packed, lptr, L, err, s) \
                 : launch_fused_r<false, W>(max_gates, X, Z, S, n, stride, nwords, packed, lptr, L, err, s);
  QS_FUSED_CASE(4)
  QS_FUSED_CASE(2)
  QS_FUSED_CASE(1)
#undef QS_FUSED_CASE
  return cudaErrorInvalidValue;
}

}  // namespace qs
