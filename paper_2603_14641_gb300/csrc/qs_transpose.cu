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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "qs_internal.cuh"

namespace qs {

// large-matrix transpose: 1024-row tiles taken row of tiles by row of tiles
// (bands of one), the fastest setting measured at 180,000 qubits in both
// directions (with 2 KB-multiple strides, 5.8 TB/s each way)
constexpr int kTransposeTileRows = 1024;
constexpr uint32_t kTransposeBand = 1;

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

// Large matrices: a persistent kernel with one 512-thread block per SM moves
// 64 KB tiles of TR input rows x 8192 / TR words with the Tensor Memory
// Accelerator: 2-D tensor-map loads bring the row segments into shared memory
// (swizzled), the block transposes the tile there in place, and 2-D stores
// send 64 (8192 / TR) output rows of TR / 64 words back. TR = 1024 (64-byte
// input and 128-byte output segments) is used; TR = 512 (128 / 64) measured
// slower at 180,000 qubits.
// Three tile buffers rotate: the load of tile k + 2 and the store of tile k - 1
// are in flight while tile k is transposed. Partial tiles at the matrix edge
// need no code: the load fills out-of-range words with zeros and the store
// drops out-of-range words.
//
// Within a tile each warp owns eight 64 x 64 sub-tiles: row blocks rt, rt + 1
// by words w0 .. w0 + 3. Lane 8 g + l holds rows 8 k + l (k = 0..7) of the
// sub-tiles of word w0 + g, so the transposition's row-index bits 5, 4, 3 are
// register indices (exchanged with byte permutes or register renaming) and
// bits 2, 1, 0 are lane bits (exchanged with shuffles inside groups of eight
// lanes). The six exchanges swap bit t of the row index with bit t of the
// column index, one t each, in any order.
constexpr int kTT = 512, kTStages = 3;
constexpr uint32_t kTileBytes = 64 * 1024;  // TR rows x TW words, TR TW = 8192
constexpr size_t kTmaSmem = (size_t)kTStages * kTileBytes + 1024 + 64;

// 16-byte chunk c of row r of a tile with rows of RB bytes (64 or 128) sits at
// chunk c ^ swz<RB>(r): the tensor map's 64- and 128-byte swizzles (address
// bits 4.. XORed with bits 7..). Callers pass r mod 8.
template <int RB>
__device__ __forceinline__ int swz(int r) { return RB == 128 ? (r & 7) : ((r >> 1) & 3); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(src)
               : "memory");
}

// exchange across lanes l and l ^ j (j = 4, 2, 1) of one 64-bit row word held
// as two halves; take / rot: the lane's bits taken from the partner and the
// left rotation that moves them into place (the lower lane of a pair takes
// the partner's bits m shifted up by j, the upper lane its bits m << j shifted
// down by j; the rotation's wrapped bits fall outside take)
__device__ __forceinline__ void xlane(uint32_t &lo, uint32_t &hi, int j, uint32_t take, uint32_t rot) {
  const uint32_t pl = __shfl_xor_sync(0xffffffffu, lo, j);
  const uint32_t ph = __shfl_xor_sync(0xffffffffu, hi, j);
  lo = (lo & ~take) | (__funnelshift_l(pl, pl, rot) & take);
  hi = (hi & ~take) | (__funnelshift_l(ph, ph, rot) & take);
}

// exchange of rows a (row-index bit clear) and b (bit set) at distance 16 or 8
// inside a thread: byte permutes of each 32-bit half
template <int J>
__device__ __forceinline__ void xreg(uint32_t &al, uint32_t &ah, uint32_t &bl, uint32_t &bh) {
  constexpr uint32_t sa = J == 16 ? 0x5410u : 0x6240u, sb = J == 16 ? 0x7632u : 0x7351u;
  const uint32_t nal = __byte_perm(al, bl, sa), nbl = __byte_perm(al, bl, sb);
  const uint32_t nah = __byte_perm(ah, bh, sa), nbh = __byte_perm(ah, bh, sb);
  al = nal; bl = nbl; ah = nah; bh = nbh;
}

// v[k] = row 8 k + l of one 64 x 64 sub-tile (l = lane & 7), as 32-bit halves
__device__ __forceinline__ void transpose_subtile(uint32_t (&vl)[8], uint32_t (&vh)[8], const uint32_t (&take)[3],
                                                  const uint32_t (&rot)[3]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // distance 32: high half of row r <-> low half of row r + 32
    const uint32_t t = vh[k];
    vh[k] = vl[k + 4];
    vl[k + 4] = t;
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if ((k & 2) == 0) xreg<16>(vl[k], vh[k], vl[k + 2], vh[k + 2]);
#pragma unroll
  for (int k = 0; k < 8; k += 2) xreg<8>(vl[k], vh[k], vl[k + 1], vh[k + 1]);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    xlane(vl[k], vh[k], 4, take[0], rot[0]);
    xlane(vl[k], vh[k], 2, take[1], rot[1]);
    xlane(vl[k], vh[k], 1, take[2], rot[2]);
  }
}

// grid: one block per SM (or fewer when there are fewer tiles); tile t of the
// tiles_x x tiles_y grid runs in block t mod gridDim.x. Tiles are numbered in
// bands of group_y tile rows, column by column inside a band, so the blocks in
// flight share both input rows and output rows.
template <int TR>
__global__ void __launch_bounds__(kTT, 1)
bit_transpose_tma_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                         uint32_t tiles_x, uint32_t tiles_y, uint32_t group_y, uint32_t out_rows,
                         uint32_t *__restrict__ err) {
  constexpr int TW = 8192 / TR, kLoadBoxes = TR / 256, kStoreBoxes = TW / 4;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kTStages * kTileBytes);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, g = lane >> 3, l = lane & 7;
  const uint64_t ntiles = (uint64_t)tiles_x * tiles_y;
  auto tile_xy = [&](uint64_t id, int &x, int &y) {
    const uint64_t band = id / ((uint64_t)group_y * tiles_x);
    const uint32_t y0 = (uint32_t)band * group_y, h = min(group_y, tiles_y - y0);
    const uint64_t rem = id - (uint64_t)y0 * tiles_x;
    x = (int)(rem / h);
    y = (int)(y0 + rem % h);
  };
  auto issue_load = [&](uint64_t id, int stage) {
    int x, y;
    tile_xy(id, x, y);
    const uint32_t bar = smem_u32(bars + stage), dst = smem_u32(base + (size_t)stage * kTileBytes);
    mbar_expect_tx(bar, kTileBytes);
#pragma unroll
    for (int q = 0; q < kLoadBoxes; ++q)
      tma_load_2d(dst + q * (kTileBytes / kLoadBoxes), &tin, TW * x, TR * y + 256 * q, bar);
  };
  if (t == 0) {
    for (int s = 0; s < kTStages; ++s) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int s = 0; s < kTStages - 1; ++s)
      if (blockIdx.x + (uint64_t)s * gridDim.x < ntiles) issue_load(blockIdx.x + (uint64_t)s * gridDim.x, s);
  }
  __syncthreads();
  // per-lane constants of the three cross-lane exchanges
  uint32_t take[3], rot[3];
  {
    const uint32_t m[3] = {0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int j = 4 >> i;
      const bool upper = (lane & j) != 0;
      take[i] = upper ? m[i] : (m[i] << j);
      rot[i] = upper ? 32 - j : j;
    }
  }
  const int rt = 2 * (warp / (TW / 4)), w = 4 * (warp % (TW / 4)) + g;
  // input rows r = 64 (rt + rb) + 8 k + l and output rows o = 64 w + 8 k + l
  // are both l mod 8, so their swizzled offsets are per-lane constants
  const int in_off = ((((w >> 1) ^ swz<TW * 8>(l)) << 1) | (w & 1));
  const int out_off = (((rt >> 1) ^ swz<TR / 8>(l)) << 1);
  bool stop = false;
  for (uint64_t k = 0, id = blockIdx.x; id < ntiles; ++k, id += gridDim.x) {
    const int stage = (int)(k % kTStages);
    const uint32_t parity = (uint32_t)((k / kTStages) & 1);
    const uint32_t bar = smem_u32(bars + stage);
    if (!mbar_try_wait(bar, parity)) {
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > 2000000000ull) { stop = true; break; }  // 2 s
    }
    uint64_t *tile = reinterpret_cast<uint64_t *>(base + (size_t)stage * kTileBytes);
    uint32_t vl[2][8], vh[2][8];
#pragma unroll
    for (int rb = 0; rb < 2; ++rb)
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint64_t v = tile[(size_t)(64 * (rt + rb) + 8 * kk + l) * TW + in_off];
        vl[rb][kk] = (uint32_t)v;
        vh[rb][kk] = (uint32_t)(v >> 32);
      }
    if (__syncthreads_or(stop)) {  // every thread leaves together
      if (t == 0) {
        atomicOr(err, kErrTimeout);
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
      }
      return;
    }
    transpose_subtile(vl[0], vh[0], take, rot);
    transpose_subtile(vl[1], vh[1], take, rot);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const size_t o = (size_t)(64 * w + 8 * kk + l);
      *reinterpret_cast<uint4 *>(tile + o * (TR / 64) + out_off) = make_uint4(vl[0][kk], vh[0][kk], vl[1][kk], vh[1][kk]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      int x, y;
      tile_xy(id, x, y);
      const uint32_t src = smem_u32(tile);
#pragma unroll
      for (int q = 0; q < kStoreBoxes; ++q)  // boxes that start past the last output row hold padding only
        if ((uint32_t)(64 * TW * x + 256 * q) < out_rows)
          tma_store_2d(&tout, (TR / 64) * y, 64 * TW * x + 256 * q, src + q * (kTileBytes / kStoreBoxes));
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      const uint64_t nid = id + (uint64_t)(kTStages - 1) * gridDim.x;
      if (nid < ntiles) {
        // the buffer of tile k - 1 takes tile k + 2 once its store has read it
        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        issue_load(nid, (int)((k + kTStages - 1) % kTStages));
      }
    }
  }
  if (t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// 2-D map of a matrix of `rows` rows x `words` 64-bit words (row stride
// `stride` words) with a box of box_w words x box_r rows
static cudaError_t word_map(CUtensorMap *m, const uint64_t *p, uint64_t words, uint64_t rows, uint64_t stride,
                            uint32_t box_w, uint32_t box_r, CUtensorMapSwizzle sw, CUtensorMapL2promotion l2) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {words, rows}, strides[1] = {stride * 8};
  const cuuint32_t box[2] = {box_w, box_r}, estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t *>(p), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, l2, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static CUtensorMapSwizzle swizzle_of(int row_bytes) {
  return row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
}

template <int TR>
static cudaError_t launch_tma_t(const uint64_t *in, size_t in_stride, size_t rows_in, size_t words_in,
                                uint64_t *out, size_t out_stride, uint32_t group_y, uint32_t *err,
                                cudaStream_t s) {
  constexpr int TW = 8192 / TR;
  static std::atomic<uint64_t> attr_set{0};
  cudaError_t e = once_per_device(attr_set, []() {
    return cudaFuncSetAttribute(bit_transpose_tma_kernel<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTmaSmem);
  });
  if (e != cudaSuccess) return e;
  // output: rows_in / 64 words per row (rows_in is a multiple of 64), 64 words_in rows
  CUtensorMap tin, tout;
  e = word_map(&tin, in, words_in, rows_in, in_stride, TW, 256, swizzle_of(TW * 8),
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B);
  if (e == cudaSuccess)
    e = word_map(&tout, out, rows_in / 64, 64 * words_in, out_stride, TR / 64, 256, swizzle_of(TR / 8),
                 CU_TENSOR_MAP_L2_PROMOTION_NONE);
  if (e != cudaSuccess) return e;
  const uint32_t tx = (uint32_t)((words_in + TW - 1) / TW), ty = (uint32_t)((rows_in + TR - 1) / TR);
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint64_t ntiles = (uint64_t)tx * ty;
  const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)sms, ntiles);
  group_y = std::max<uint32_t>(1, std::min(group_y, ty));
  bit_transpose_tma_kernel<TR><<<grid, kTT, kTmaSmem, s>>>(tin, tout, tx, ty, group_y,
                                                           (uint32_t)(64 * words_in), err);
  return cudaGetLastError();
}

// tile_rows: 512 (128-byte input / 64-byte output segments) or 1024 (64 / 128)
cudaError_t launch_transpose_tma(const uint64_t *in, size_t in_stride, size_t rows_in, size_t words_in,
                                 uint64_t *out, size_t out_stride, int tile_rows, uint32_t group_y,
                                 uint32_t *err, cudaStream_t s) {
  if (tile_rows == 1024)
    return launch_tma_t<1024>(in, in_stride, rows_in, words_in, out, out_stride, group_y, err, s);
  return launch_tma_t<512>(in, in_stride, rows_in, words_in, out, out_stride, group_y, err, s);
}

static cudaError_t transpose(const uint64_t *in, size_t in_stride, size_t rows_in, size_t words_in,
                             uint64_t *out, size_t out_stride, uint32_t band, uint32_t *err, cudaStream_t s) {
  if (rows_in >= 512 && words_in >= 16)
    return launch_transpose_tma(in, in_stride, rows_in, words_in, out, out_stride, kTransposeTileRows, band,
                                err, s);
  // rows_in is a multiple of 256 and words_in of 4 by construction
  dim3 grid((unsigned)(words_in / 4), (unsigned)(rows_in / 256));
  bit_transpose_kernel<<<grid, 128, 0, s>>>(in, in_stride, out, out_stride);
  return cudaGetLastError();
}

cudaError_t launch_to_rows(const Dev &d, cudaStream_t s) {
  // in = X/Z: rows = ncols (qubits), words = cs; out = RX/RZ: rows = 64 cs, words = rs
  const Layout &L = d.L;
  cudaError_t e = transpose(d.X, L.cs, L.ncols, L.cs, d.RX, L.rs, kTransposeBand, d.err, s);
  if (e == cudaSuccess) e = transpose(d.Z, L.cs, L.ncols, L.cs, d.RZ, L.rs, kTransposeBand, d.err, s);
  return e;
}

cudaError_t launch_to_cols(const Dev &d, cudaStream_t s) {
  // in = RX/RZ: rows = 64 cs, words = rs; out = X/Z: rows = 64 rs = ncols, words = cs
  const Layout &L = d.L;
  cudaError_t e = transpose(d.RX, L.rs, L.nrows, L.rs, d.X, L.cs, kTransposeBand, d.err, s);
  if (e == cudaSuccess) e = transpose(d.RZ, L.rs, L.nrows, L.rs, d.Z, L.cs, kTransposeBand, d.err, s);
  return e;
}

}  // namespace qs
