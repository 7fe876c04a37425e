// Layout change between the column-major tableau (gate layers) and the
// row-major tableau (measurement), Sec. 4.5 (Alg. 4).
//
// The paper transposes in place with a shared-memory tile shuffle plus an
// off-diagonal swap. With 280 GB of HBM the row-major copy lives in its own
// buffers, so the transpose here is out of place and does one read and one
// write of each word. One generic kernel serves both directions: it reads a
// bit matrix M stored as `in` rows of words (bit b of in[i][j] = M[i][64 j + b])
// and writes M^T the same way.
//
// Small matrices: a block is four warps and covers 256 input rows x 4 input
// words:
//   - lane l of warp w loads input rows 64 w + l and 64 w + l + 32, 4 words
//     each (one full 32-byte sector per row);
//   - each 64 x 64 bit sub-tile is transposed in registers in six
//     mask/shift rounds: the first between the lane's two rows, the other
//     five between lanes l and l ^ j with warp shuffles (the bit-group swap
//     of Alg. 4 with its six masks, done in registers);
//   - the transposed words meet in shared memory and leave as 32-byte output
//     row segments.
#include "qs_internal.cuh"

namespace qs {

__device__ __forceinline__ void transpose64(uint64_t &lo, uint64_t &hi, int lane) {
  // rows lane (lo) and lane + 32 (hi); after the call lo/hi hold output rows
  // lane and lane + 32 (bit a of output row b = bit b of input row a).
  {
    const uint64_t m = 0x00000000FFFFFFFFull;
    uint64_t t = ((lo >> 32) ^ hi) & m;
    lo ^= t << 32;
    hi ^= t;
  }
  const uint64_t masks[5] = {0x0000FFFF0000FFFFull, 0x00FF00FF00FF00FFull, 0x0F0F0F0F0F0F0F0Full,
                             0x3333333333333333ull, 0x5555555555555555ull};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint64_t m = masks[s];
    uint64_t plo = __shfl_xor_sync(0xffffffffu, lo, j);
    uint64_t phi = __shfl_xor_sync(0xffffffffu, hi, j);
    if ((lane & j) == 0) {
      uint64_t t = ((lo >> j) ^ plo) & m;
      lo ^= t << j;
      t = ((hi >> j) ^ phi) & m;
      hi ^= t << j;
    } else {
      uint64_t t = ((plo >> j) ^ lo) & m;
      lo ^= t;
      t = ((phi >> j) ^ hi) & m;
      hi ^= t;
    }
  }
}

// in:  rows_in x words_in (stride in_stride words); out: rows_out x words_out
// grid.x = words_in / 4, grid.y = rows_in / 256 (both exact by construction)
__global__ void __launch_bounds__(128)
bit_transpose_kernel(const uint64_t *__restrict__ in, size_t in_stride, uint64_t *__restrict__ out,
                     size_t out_stride) {
  __shared__ uint64_t tile[256][5];  // [output row within block][output word], padded
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t j0 = (size_t)blockIdx.x * 4;        // input word group
  const size_t i0 = (size_t)blockIdx.y * 256;      // input row group
  const size_t r0 = i0 + 64 * warp + lane;
  const ulonglong2 *p0 = reinterpret_cast<const ulonglong2 *>(in + r0 * in_stride + j0);
  const ulonglong2 *p1 = reinterpret_cast<const ulonglong2 *>(in + (r0 + 32) * in_stride + j0);
  ulonglong2 a0 = p0[0], a1 = p0[1], b0 = p1[0], b1 = p1[1];
  uint64_t lo[4] = {a0.x, a0.y, a1.x, a1.y};
  uint64_t hi[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    transpose64(lo[s], hi[s], lane);
    // sub-tile (input word j0 + s, input rows i0 + 64 warp ..): output rows
    // 64 (j0 + s) + b, output word i0 / 64 + warp
    tile[64 * s + lane][warp] = lo[s];
    tile[64 * s + lane + 32][warp] = hi[s];
  }
  __syncthreads();
  // 256 output rows x 4 words: thread t writes rows t and t + 128
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int rr = threadIdx.x + 128 * h;
    const size_t orow = 64 * j0 + rr;
    ulonglong2 *q = reinterpret_cast<ulonglong2 *>(out + orow * out_stride + i0 / 64);
    q[0] = make_ulonglong2(tile[rr][0], tile[rr][1]);
    q[1] = make_ulonglong2(tile[rr][2], tile[rr][3]);
  }
}

// Branch-free form of transpose64 for the large-matrix kernel. In the round of
// distance j the lower lane of a pair keeps its bits outside m << j and takes
// its partner's bits m, shifted up by j; the upper lane keeps its bits outside m
// and takes its partner's bits m << j, shifted down. Both are one bit-select
// of a value shifted the lane's way, so no lane-dependent branch remains (the
// two sides of that branch used to run one after the other).
__device__ __forceinline__ void transpose64_sel(uint64_t &lo, uint64_t &hi, int lane) {
  {
    const uint64_t m = 0x00000000FFFFFFFFull;
    uint64_t t = ((lo >> 32) ^ hi) & m;
    lo ^= t << 32;
    hi ^= t;
  }
  const uint64_t masks[5] = {0x0000FFFF0000FFFFull, 0x00FF00FF00FF00FFull, 0x0F0F0F0F0F0F0F0Full,
                             0x3333333333333333ull, 0x5555555555555555ull};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint64_t m = masks[s];
    const bool upper = (lane & j) != 0;
    const uint64_t take = upper ? m : (m << j);  // bits taken from the partner
    const uint64_t plo = __shfl_xor_sync(0xffffffffu, lo, j);
    const uint64_t phi = __shfl_xor_sync(0xffffffffu, hi, j);
    const uint64_t slo = upper ? (plo >> j) : (plo << j);
    const uint64_t shi = upper ? (phi >> j) : (phi << j);
    lo = (lo & ~take) | (slo & take);
    hi = (hi & ~take) | (shi & take);
  }
}

// Large matrices: a block of 512 threads covers 512 input rows x 16 input
// words, so reads are 128-byte row segments and writes 64-byte ones (32-byte
// segments reach only about a third of the HBM bandwidth). The tile is staged
// in shared memory (70 KB, three blocks per SM overlap their load, transpose
// and store phases), each warp transposes 64 x 64 sub-tiles in registers and
// writes them back in place, and 1024 output rows of 8 words leave the
// block. Row stride 17 words and an XOR swizzle of the word index by the
// 64-row group keep the three shared-memory passes free of bank conflicts.
// Partial tiles at the matrix edge read zeros and write only in-range words.
constexpr int kTR = 512, kTW = 16, kTP = 17, kTT = 512;  // rows, words, row stride, threads
constexpr size_t kBigTileSmem = (size_t)kTR * kTP * sizeof(uint64_t);

__device__ __forceinline__ int tsw(int row, int w) { return row * kTP + (w ^ (row >> 6)); }

__global__ void __launch_bounds__(kTT, 3)
bit_transpose_big_kernel(const uint64_t *__restrict__ in, size_t in_stride, size_t rows_in,
                         size_t words_in, uint64_t *__restrict__ out, size_t out_stride) {
  extern __shared__ uint64_t tl[];  // [kTR][kTP], word index swizzled
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const size_t i0 = (size_t)blockIdx.y * kTR, j0 = (size_t)blockIdx.x * kTW;
  const int vr = (int)min((size_t)kTR, rows_in - i0), vw = (int)min((size_t)kTW, words_in - j0);
  // 1: 16 words of a row per 8 threads, two words each (128-byte segments)
#pragma unroll 4
  for (int it = 0; it < kTR * kTW / (2 * kTT); ++it) {
    const int idx = it * kTT + t, row = idx / (kTW / 2), w = 2 * (idx % (kTW / 2));
    ulonglong2 v = make_ulonglong2(0, 0);
    if (row < vr && w + 1 < vw) {
      v = *reinterpret_cast<const ulonglong2 *>(in + (i0 + row) * in_stride + j0 + w);
    } else if (row < vr && w < vw) {
      v.x = in[(i0 + row) * in_stride + j0 + w];
    }
    tl[tsw(row, w)] = v.x;
    tl[tsw(row, w + 1)] = v.y;
  }
  __syncthreads();
  // 2: 256 sub-tiles (16 row groups x 16 words), 8 per warp
#pragma unroll 1
  for (int k = 0; k < (kTR / 64) * kTW / (kTT / 32); ++k) {
    const int st = warp * ((kTR / 64) * kTW / (kTT / 32)) + k, rt = st / kTW, w = st % kTW;
    uint64_t lo = tl[tsw(64 * rt + lane, w)], hi = tl[tsw(64 * rt + lane + 32, w)];
    transpose64_sel(lo, hi, lane);
    // now lo = output row 64 w + lane, word rt; hi = output row 64 w + lane + 32
    tl[tsw(64 * rt + lane, w)] = lo;
    tl[tsw(64 * rt + lane + 32, w)] = hi;
  }
  __syncthreads();
  // 3: output row 64 w + b, word rt sits at [64 rt + b][w]; kTR / 64 words per output row
  const int vrt = vr / 64;  // rows_in is a multiple of 64
#pragma unroll 4
  for (int it = 0; it < kTR * kTW / kTT; ++it) {
    const int idx = it * kTT + t, orl = idx / (kTR / 64), rt = idx % (kTR / 64);
    const int w = orl / 64, b = orl % 64;
    if (w < vw && rt < vrt)
      out[(64 * (j0 + w) + b) * out_stride + i0 / 64 + rt] = tl[tsw(64 * rt + b, w)];
  }
}

static std::atomic<uint64_t> g_big_tile_attr{0};

static cudaError_t transpose(const uint64_t *in, size_t in_stride, size_t rows_in, size_t words_in,
                             uint64_t *out, size_t out_stride, cudaStream_t s) {
  if (rows_in >= (size_t)kTR && words_in >= (size_t)kTW) {
    cudaError_t e = once_per_device(g_big_tile_attr, []() {
      return cudaFuncSetAttribute(bit_transpose_big_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBigTileSmem);
    });
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((words_in + kTW - 1) / kTW), (unsigned)((rows_in + kTR - 1) / kTR));
    bit_transpose_big_kernel<<<grid, kTT, kBigTileSmem, s>>>(in, in_stride, rows_in, words_in, out,
                                                               out_stride);
  } else {
    // rows_in is a multiple of 256 and words_in of 4 by construction
    dim3 grid((unsigned)(words_in / 4), (unsigned)(rows_in / 256));
    bit_transpose_kernel<<<grid, 128, 0, s>>>(in, in_stride, out, out_stride);
  }
  return cudaGetLastError();
}

cudaError_t launch_to_rows(const Dev &d, cudaStream_t s) {
  // in = X/Z: rows = ncols (qubits), words = cs; out = RX/RZ: rows = 64 cs, words = rs
  const Layout &L = d.L;
  cudaError_t e = transpose(d.X, L.cs, L.ncols, L.cs, d.RX, L.rs, s);
  if (e == cudaSuccess) e = transpose(d.Z, L.cs, L.ncols, L.cs, d.RZ, L.rs, s);
  return e;
}

cudaError_t launch_to_cols(const Dev &d, cudaStream_t s) {
  // in = RX/RZ: rows = 64 cs, words = rs; out = X/Z: rows = 64 rs = ncols, words = cs
  const Layout &L = d.L;
  cudaError_t e = transpose(d.RX, L.rs, L.nrows, L.rs, d.X, L.cs, s);
  if (e == cudaSuccess) e = transpose(d.RZ, L.rs, L.nrows, L.rs, d.Z, L.cs, s);
  return e;
}

}  // namespace qs
