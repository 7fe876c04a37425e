// Batched persistent launch: many independent circuits of uneven size in ONE
// kernel launch.
//
// The paper simulates one circuit at a time with one kernel per window and a
// host loop over measurements (Sec. 4.1, Alg. 2). Small circuits leave most of
// a GB300 idle and pay a launch per step. Here a cooperative persistent kernel
// walks every circuit's program in lock-step rounds (a round = a segment of gate
// layers followed by a list of Z-measurements) and spreads each phase of a round
// over all CTAs through flattened work lists (a work queue built on the host
// from the circuits' sizes; items are taken grid-stride):
//   init      zero X/Z/S, set D_i = X_i, S_i = Z_i               (Alg. 2 init)
//   gates     (circuit, column word) slices in shared memory, every layer of
//             the round applied there (rows are independent, Sec. 2.4)
//   to rows   64x64 bit-tile transposes (Sec. 4.5)
//   for measurement j of the round, over circuits that have a j-th one:
//     A  gather column q, pivot by atomicMin                    (Sec. 2.5)
//     B  rowsum into anticommuting rows, or deterministic-product chunks
//     C  finalize (D_{p-n} <- S_p, S_p <- (-1)^b Z_q) or combine chunks; record
//   to cols   transposes back for the next round's gates
// Phases are separated by a grid barrier whose spin is bounded: when it runs out
// the kernel sets the timeout flag and every CTA returns (no hang).
// Semantics are exactly those of the single-circuit path (qs_sim_*), so a
// circuit's record and tableau are bit-identical alone and in a batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <thread>
#include <climits>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qs_internal.cuh"
#include "qs_rules.cuh"

namespace qs {

constexpr int64_t kBNoPivot = LLONG_MAX;
constexpr uint32_t kBatchMaxQubits = 8192;  // det partials: <= 4 words per lane
// Circuits of at least this many qubits run through per-circuit simulators
// (blocked measurement, 64 measurements per tableau pass) on worker streams;
// the persistent kernel takes the smaller ones, whose per-launch costs
// dominate when they run alone.
constexpr uint32_t kBatchSimMinQubits = 1024;
constexpr uint32_t kBatchMaxWorkers = 16;
constexpr uint32_t kBatchLimitQubits = 1u << 20;

struct BCirc {
  uint32_t n, k, cs, rs, ncols, nrows;
  uint32_t lpr, pad_;  // lanes per row in the update phase (power of two <= 32)
  uint64_t *X, *Z, *S, *RX, *RZ;
  uint32_t *colx;
  int64_t *mst;
  uint64_t *det_x, *det_z;  // k chunks x rs words
  int32_t *det_scal;        // k
  const uint32_t *gates;    // packed records of this circuit
  const int64_t *lptr;      // n_layers + 1 offsets into gates
  const uint32_t *qubits;   // measured qubits in program order
  uint8_t *record;
  uint64_t seed, shot;
};

struct BAct {
  uint32_t c, l0, l1, q0, qn, pad;
  uint64_t m0;    // record index of the round's first measurement
  uint64_t pre;   // exclusive prefix of the list's items (slices / tiles)
  uint64_t pre2;  // exclusive prefix of rows (measurement list)
  uint64_t pre3;  // exclusive prefix of warp units (32 / lpr rows each) in the update phase
};

struct BRound {
  uint32_t g_first, g_count, m_first, m_count, max_qn, pad;
};

struct BProg {
  const BCirc *circs;
  const BAct *acts;
  const BRound *rounds;
  const uint64_t *pre_n;
  uint64_t *zero_begin;
  uint64_t zero_words, spin_limit;
  uint32_t ncirc, nrounds, wpb, fuse_depth;
  uint32_t *bar, *err;
};

__device__ __forceinline__ int bmod4(int v) { return ((v % 4) + 4) % 4; }

// bounded grid barrier (all CTAs are co-resident: cooperative launch)
__device__ bool grid_sync(const BProg &P) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t *vgen = P.bar + 1;
    volatile uint32_t *verr = P.err;
    const uint32_t gen = *vgen;
    __threadfence();
    const uint32_t arrived = atomicAdd(P.bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(P.bar, 0u);
      __threadfence();
      atomicAdd(P.bar + 1, 1u);
    } else {
      uint64_t it = 0;
      while (*vgen == gen) {
        if (*verr & kErrTimeout) { ok = 0; break; }
        if (++it > P.spin_limit) { atomicOr(P.err, kErrTimeout); ok = 0; break; }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = ok && !(*verr & kErrTimeout);
  }
  __syncthreads();
  return s_ok != 0;
}

// entry of a list [first, first + count) holding flattened index i
__device__ __forceinline__ uint32_t find_act(const BAct *a, uint32_t first, uint32_t count,
                                             uint64_t i, int key) {
  uint32_t lo = 0, hi = count;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint64_t v = key == 2 ? a[first + mid].pre3 : (key == 1 ? a[first + mid].pre2 : a[first + mid].pre);
    if (v <= i) lo = mid; else hi = mid;
  }
  return first + lo;
}

__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}

// one 256-row x 4-word tile of a bit-matrix transpose by a 128-thread group
// (same arithmetic as bit_transpose_kernel)
__device__ void transpose_tile(const uint64_t *in, size_t in_stride, uint64_t *out,
                               size_t out_stride, size_t j0, size_t i0, uint64_t (*tile)[5],
                               int gthread, int gid) {
  const int lane = gthread & 31, warp = gthread >> 5;
  const size_t r0 = i0 + 64 * warp + lane;
  const ulonglong2 *p0 = reinterpret_cast<const ulonglong2 *>(in + r0 * in_stride + j0);
  const ulonglong2 *p1 = reinterpret_cast<const ulonglong2 *>(in + (r0 + 32) * in_stride + j0);
  ulonglong2 a0 = p0[0], a1 = p0[1], b0 = p1[0], b1 = p1[1];
  uint64_t lo[4] = {a0.x, a0.y, a1.x, a1.y};
  uint64_t hi[4] = {b0.x, b0.y, b1.x, b1.y};
  const uint64_t masks[5] = {0x0000FFFF0000FFFFull, 0x00FF00FF00FF00FFull, 0x0F0F0F0F0F0F0F0Full,
                             0x3333333333333333ull, 0x5555555555555555ull};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    uint64_t l = lo[s], h = hi[s];
    {
      uint64_t t = ((l >> 32) ^ h) & 0x00000000FFFFFFFFull;
      l ^= t << 32;
      h ^= t;
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int j = 16 >> r;
      const uint64_t m = masks[r];
      const uint64_t pl = __shfl_xor_sync(0xffffffffu, l, j), ph = __shfl_xor_sync(0xffffffffu, h, j);
      if ((lane & j) == 0) {
        l ^= (((l >> j) ^ pl) & m) << j;
        h ^= (((h >> j) ^ ph) & m) << j;
      } else {
        l ^= ((pl >> j) ^ l) & m;
        h ^= ((ph >> j) ^ h) & m;
      }
    }
    tile[64 * s + lane][warp] = l;
    tile[64 * s + lane + 32][warp] = h;
  }
  group_bar(gid);
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const int rr = gthread + 128 * hh;
    ulonglong2 *q = reinterpret_cast<ulonglong2 *>(out + (64 * j0 + rr) * out_stride + i0 / 64);
    q[0] = make_ulonglong2(tile[rr][0], tile[rr][1]);
    q[1] = make_ulonglong2(tile[rr][2], tile[rr][3]);
  }
  group_bar(gid);
}

__device__ void phase_transpose(const BProg &P, const BRound &R, bool to_rows, uint64_t *smem) {
  const uint32_t groups = blockDim.x / 128;
  const int gid = threadIdx.x / 128, gthread = threadIdx.x % 128;
  uint64_t(*tile)[5] = reinterpret_cast<uint64_t(*)[5]>(smem + (size_t)gid * 256 * 5);
  const uint64_t total = P.acts[R.m_first + R.m_count].pre;
  for (uint64_t t = (uint64_t)blockIdx.x * groups + gid; t < total; t += (uint64_t)gridDim.x * groups) {
    const BAct &A = P.acts[find_act(P.acts, R.m_first, R.m_count, t, 0)];
    const BCirc &C = P.circs[A.c];
    const uint64_t per = (uint64_t)(C.cs / 4) * (C.ncols / 256);
    const uint64_t tt = t - A.pre;
    const bool zmat = tt >= per;
    const uint64_t u = zmat ? tt - per : tt;
    if (to_rows) {
      const uint32_t gx = C.cs / 4;
      transpose_tile(zmat ? C.Z : C.X, C.cs, zmat ? C.RZ : C.RX, C.rs, 4 * (u % gx), 256 * (u / gx),
                     tile, gthread, gid + 1);
    } else {
      const uint32_t gx = C.rs / 4;
      transpose_tile(zmat ? C.RZ : C.RX, C.rs, zmat ? C.Z : C.X, C.cs, 4 * (u % gx), 256 * (u / gx),
                     tile, gthread, gid + 1);
    }
  }
}

__device__ void phase_gates(const BProg &P, const BRound &R, uint64_t *smem) {
  const uint64_t total = P.acts[R.g_first + R.g_count].pre;
  const uint32_t W = P.wpb;
  for (uint64_t it = blockIdx.x; it < total; it += gridDim.x) {
    const BAct &A = P.acts[find_act(P.acts, R.g_first, R.g_count, it, 0)];
    const BCirc &C = P.circs[A.c];
    const uint32_t n = C.n, w0 = (uint32_t)(it - A.pre) * W;
    uint64_t *sx = smem, *sz = smem + (size_t)n * W;
    const uint32_t depth = P.fuse_depth ? P.fuse_depth : (A.l1 - A.l0);
    uint64_t sacc[2] = {0, 0};
    for (uint32_t lb = A.l0; lb < A.l1; lb += depth) {
      const uint32_t le = min(A.l1, lb + depth);
      for (uint32_t q = threadIdx.x; q < n; q += blockDim.x)
        for (uint32_t j = 0; j < W; ++j) {
          const bool in = w0 + j < C.cs;
          sx[q * W + j] = in ? C.X[(size_t)q * C.cs + w0 + j] : 0ull;
          sz[q * W + j] = in ? C.Z[(size_t)q * C.cs + w0 + j] : 0ull;
        }
      __syncthreads();
      for (uint32_t l = lb; l < le; ++l) {
        const int64_t g1 = C.lptr[l + 1];
        for (int64_t g = C.lptr[l] + threadIdx.x; g < g1; g += blockDim.x) {
          const uint32_t wd = __ldg(C.gates + 2 * g), qb = __ldg(C.gates + 2 * g + 1);
          const uint32_t type = wd >> 24, qa = wd & 0xFFFFFFu;
          const bool two = type >= QS_CX && type <= QS_ISWAP;
          if (qa >= n || type >= QS_NUM_GATE_TYPES || (two && (qb >= n || qb == qa))) {
            atomicOr(P.err, kErrBadGate);
            continue;
          }
          for (uint32_t j = 0; j < W; ++j) {
            uint64_t xa = sx[qa * W + j], za = sz[qa * W + j], xb = 0, zb = 0;
            if (two) { xb = sx[qb * W + j]; zb = sz[qb * W + j]; }
            rule<true>(type, xa, za, xb, zb, sacc[j]);
            sx[qa * W + j] = xa;
            sz[qa * W + j] = za;
            if (two) { sx[qb * W + j] = xb; sz[qb * W + j] = zb; }
          }
        }
        __syncthreads();
      }
      for (uint32_t q = threadIdx.x; q < n; q += blockDim.x)
        for (uint32_t j = 0; j < W; ++j)
          if (w0 + j < C.cs) {
            C.X[(size_t)q * C.cs + w0 + j] = sx[q * W + j];
            C.Z[(size_t)q * C.cs + w0 + j] = sz[q * W + j];
          }
      __syncthreads();
    }
    // block XOR of the sign words
    __shared__ uint64_t red[2][32];
    for (uint32_t j = 0; j < W; ++j) {
      uint64_t v = sacc[j];
      for (int o = 16; o > 0; o >>= 1) v ^= __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < W && w0 + threadIdx.x < C.cs) {
      uint64_t v = 0;
      for (uint32_t wp = 0; wp < blockDim.x / 32; ++wp) v ^= red[threadIdx.x][wp];
      C.S[w0 + threadIdx.x] ^= v;
    }
    __syncthreads();
  }
}

// number of measure-list entries (sorted by qn, descending) with qn > j
__device__ __forceinline__ uint32_t active_count(const BProg &P, const BRound &R, uint32_t j) {
  uint32_t lo = 0, hi = R.m_count;  // first index with qn <= j
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (P.acts[R.m_first + mid].qn > j) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// contiguous range [*b, *e) of `total` items for the calling warp
__device__ __forceinline__ void warp_range(uint64_t total, uint64_t *b, uint64_t *e) {
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t per = (total + nw - 1) / nw;
  *b = min(total, w * per);
  *e = min(total, *b + per);
}

__device__ void phase_gather(const BProg &P, const BRound &R, uint32_t j, uint32_t a) {
  // a warp takes a contiguous run of 32-row groups; circuits are found once
  // per run and then followed linearly
  const uint64_t groups = P.acts[R.m_first + a].pre2 >> 5;
  uint64_t g0, g1;
  warp_range(groups, &g0, &g1);
  if (g0 >= g1) return;
  const int lane = threadIdx.x & 31;
  uint32_t e = find_act(P.acts, R.m_first, a, g0 << 5, 1);
  for (uint64_t g = g0; g < g1; ++g) {
    const uint64_t i = g << 5;
    while (e + 1 < R.m_first + a && P.acts[e + 1].pre2 <= i) ++e;
    const BAct &A = P.acts[e];
    const BCirc &C = P.circs[A.c];
    const uint32_t r = (uint32_t)(i - A.pre2) + lane;
    const uint32_t q = C.qubits[A.q0 + j];
    uint32_t bit = 0;
    if (q < C.n) bit = (uint32_t)(C.RX[(size_t)r * C.rs + (q >> 6)] >> (q & 63)) & 1u;
    const uint32_t ball = __ballot_sync(0xffffffffu, bit);
    if (lane == 0) {
      if (q >= C.n) {
        if (r == 0) atomicOr(P.err, kErrBadQubit);
        continue;
      }
      C.colx[r >> 5] = ball;
      const uint64_t lo = 64ull * C.k, hi = 64ull * C.k + C.n, base = r;
      uint32_t m = ball;
      if (base + 32 > lo && base < hi && m) {
        if (base < lo) m &= ~0u << (uint32_t)(lo - base);
        if (base + 32 > hi) m &= (uint32_t)((1ull << (hi - base)) - 1);
        if (m) atomicMin(reinterpret_cast<long long *>(&C.mst[kMsPivot]), (long long)(base + __ffs(m) - 1));
      }
    }
  }
}

__device__ void phase_update(const BProg &P, const BRound &R, uint32_t j, uint32_t a) {
  // warp units: a unit is 32 / lpr consecutive rows of one circuit, lpr lanes per row
  const uint64_t total = P.acts[R.m_first + a].pre3;
  const int lane = threadIdx.x & 31;
  uint64_t u0, u1;
  warp_range(total, &u0, &u1);
  if (u0 >= u1) return;
  uint32_t e = find_act(P.acts, R.m_first, a, u0, 2);
  for (uint64_t i = u0; i < u1; ++i) {
    while (e + 1 < R.m_first + a && P.acts[e + 1].pre3 <= i) ++e;
    const BAct &A = P.acts[e];
    const BCirc &C = P.circs[A.c];
    const uint32_t G = C.lpr, rpw = 32 / G;
    const uint32_t unit = (uint32_t)(i - A.pre3);
    const uint32_t q = C.qubits[A.q0 + j];
    if (q >= C.n) continue;
    const int64_t p = C.mst[kMsPivot];
    if (p != kBNoPivot) {
      const int64_t pd = p - 64ll * C.k;
      const uint32_t sub = lane / G, sl = lane % G;
      const uint32_t r = unit * rpw + sub;
      const bool tgt = r < C.nrows && ((C.colx[r >> 5] >> (r & 31)) & 1u) != 0 && (int64_t)r != p &&
                       (int64_t)r != pd;
      int acc = 0;
      if (tgt) {
        const ulonglong2 *px = reinterpret_cast<const ulonglong2 *>(C.RX + (size_t)p * C.rs);
        const ulonglong2 *pz = reinterpret_cast<const ulonglong2 *>(C.RZ + (size_t)p * C.rs);
        ulonglong2 *rx = reinterpret_cast<ulonglong2 *>(C.RX + (size_t)r * C.rs);
        ulonglong2 *rz = reinterpret_cast<ulonglong2 *>(C.RZ + (size_t)r * C.rs);
        for (uint32_t v = sl; v < C.rs / 2; v += G) {
          const ulonglong2 x = rx[v], z = rz[v], ax = px[v], cz = pz[v];
          const ulonglong2 nx = make_ulonglong2(x.x ^ ax.x, x.y ^ ax.y);
          const ulonglong2 nz = make_ulonglong2(z.x ^ cz.x, z.y ^ cz.y);
          acc += __popcll(x.x & z.x) + __popcll(x.y & z.y);
          acc += 2 * (__popcll(cz.x & x.x) + __popcll(cz.y & x.y));
          acc += __popcll(ax.x & cz.x) + __popcll(ax.y & cz.y);  // |x_p & z_p| for this word
          acc -= __popcll(nx.x & nz.x) + __popcll(nx.y & nz.y);
          rx[v] = nx;
          rz[v] = nz;
        }
      }
      // reduction inside each group of G lanes (offsets < G never cross groups)
      for (uint32_t o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (sl == 0 && tgt) {
        const int rp = (int)((C.S[p >> 6] >> (p & 63)) & 1u);
        const int t = bmod4(acc + 2 * rp);
        if (t & 1) atomicOr(P.err, kErrOddPhase);
        if (t >> 1) atomicXor(reinterpret_cast<unsigned long long *>(&C.S[r >> 6]), 1ull << (r & 63));
      }
    } else {
      // deterministic case: chunks (64 destabilizer rows each) of this unit, whole warp per chunk
      const uint64_t *colx64 = reinterpret_cast<const uint64_t *>(C.colx);
      for (uint32_t r = unit * rpw; r < (unit + 1) * rpw && r < C.k; ++r) {
        uint64_t m = colx64[r];
        uint64_t px[4] = {0, 0, 0, 0}, pz[4] = {0, 0, 0, 0}, cross = 0;
        int cnt = 0;
        const int rsum = __popcll(m & C.S[C.k + r]);
        while (m) {
          const int b = __ffsll((long long)m) - 1;
          m &= m - 1;
          const size_t row = 64ull * C.k + 64ull * r + b;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const uint32_t u = lane + 32 * t;
            if (u < C.k) {
              const uint64_t x = C.RX[row * C.rs + u], z = C.RZ[row * C.rs + u];
              cross ^= x & pz[t];
              cnt += __popcll(x & z);
              px[t] ^= x;
              pz[t] ^= z;
            }
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t u = lane + 32 * t;
          if (u < C.k) {
            C.det_x[(size_t)r * C.rs + u] = px[t];
            C.det_z[(size_t)r * C.rs + u] = pz[t];
          }
        }
        int v = cnt + 2 * (__popcll(cross) & 1);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) C.det_scal[r] = bmod4(v + 2 * rsum);
      }
    }
  }
}

__device__ void phase_finalize(const BProg &P, const BRound &R, uint32_t j, uint32_t a) {
  __shared__ int s_par, s_bad;
  for (uint32_t e = blockIdx.x; e < a; e += gridDim.x) {
    const BAct &A = P.acts[R.m_first + e];
    const BCirc &C = P.circs[A.c];
    const uint32_t q = C.qubits[A.q0 + j];
    const uint64_t midx = A.m0 + j;
    const int64_t p = C.mst[kMsPivot];
    __syncthreads();
    if (q >= C.n) {
      if (threadIdx.x == 0) { C.record[midx] = 0; C.mst[kMsPivot] = kBNoPivot; }
      __syncthreads();
      continue;
    }
    if (p != kBNoPivot) {
      const int64_t pd = p - 64ll * C.k;
      for (uint32_t u = threadIdx.x; u < C.rs; u += blockDim.x) {
        const uint64_t x = C.RX[(size_t)p * C.rs + u], z = C.RZ[(size_t)p * C.rs + u];
        C.RX[(size_t)pd * C.rs + u] = x;
        C.RZ[(size_t)pd * C.rs + u] = z;
        C.RX[(size_t)p * C.rs + u] = 0;
        C.RZ[(size_t)p * C.rs + u] = (u == (q >> 6)) ? (1ull << (q & 63)) : 0ull;
      }
      if (threadIdx.x == 0) {
        const uint32_t b = (uint32_t)(philox4x64_10(midx, C.shot, 0, 0, C.seed, kCoinKey).v[0] & 1u);
        const uint64_t sp = (C.S[p >> 6] >> (p & 63)) & 1u;
        C.S[pd >> 6] = (C.S[pd >> 6] & ~(1ull << (pd & 63))) | (sp << (pd & 63));
        C.S[p >> 6] = (C.S[p >> 6] & ~(1ull << (p & 63))) | ((uint64_t)b << (p & 63));
        C.record[midx] = (uint8_t)b;
      }
    } else {
      if (threadIdx.x == 0) { s_par = 0; s_bad = 0; }
      __syncthreads();
      for (uint32_t u = threadIdx.x; u < C.k; u += blockDim.x) {
        uint64_t cross = 0, xb = 0, zb = 0;
        for (uint32_t b = 0; b < C.k; ++b) {
          const uint64_t x = C.det_x[(size_t)b * C.rs + u], z = C.det_z[(size_t)b * C.rs + u];
          cross ^= x & zb;
          xb ^= x;
          zb ^= z;
        }
        const uint64_t want = (u == (q >> 6)) ? (1ull << (q & 63)) : 0ull;
        if (__popcll(cross) & 1) atomicXor(&s_par, 1);
        if (xb != 0 || zb != want) atomicOr(&s_bad, 1);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 2 * s_par;
        for (uint32_t b = 0; b < C.k; ++b) t += C.det_scal[b];
        t = bmod4(t);
        if ((t & 1) || s_bad) atomicOr(P.err, s_bad ? kErrDetProduct : kErrOddPhase);
        C.record[midx] = (uint8_t)(t >> 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) C.mst[kMsPivot] = kBNoPivot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) batch_kernel(BProg P, uint32_t round_limit) {
  extern __shared__ uint64_t smem[];
  const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  // init: zero X, Z, S of every circuit, then the identity tableau
  for (uint64_t i = gt; i < P.zero_words; i += nt) P.zero_begin[i] = 0;
  if (!grid_sync(P)) return;
  const uint64_t nq = P.pre_n[P.ncirc];
  for (uint64_t i = gt; i < nq; i += nt) {
    uint32_t lo = 0, hi = P.ncirc;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (P.pre_n[mid] <= i) lo = mid; else hi = mid;
    }
    const BCirc &C = P.circs[lo];
    const uint32_t q = (uint32_t)(i - P.pre_n[lo]);
    C.X[(size_t)q * C.cs + (q >> 6)] = 1ull << (q & 63);
    C.Z[(size_t)q * C.cs + C.k + (q >> 6)] = 1ull << (q & 63);
    if (q == 0)
      for (int w = 0; w < kMeasStateWords; ++w) C.mst[w] = (w == kMsPivot) ? kBNoPivot : 0;
  }
  if (!grid_sync(P)) return;
  const uint32_t nr = min(P.nrounds, round_limit);
  for (uint32_t r = 0; r < nr; ++r) {
    const BRound R = P.rounds[r];
    if (R.g_count) {
      phase_gates(P, R, smem);
      if (!grid_sync(P)) return;
    }
    if (R.m_count) {
      phase_transpose(P, R, true, smem);
      if (!grid_sync(P)) return;
      for (uint32_t j = 0; j < R.max_qn; ++j) {
        const uint32_t a = active_count(P, R, j);
        phase_gather(P, R, j, a);
        if (!grid_sync(P)) return;
        phase_update(P, R, j, a);
        if (!grid_sync(P)) return;
        phase_finalize(P, R, j, a);
        if (!grid_sync(P)) return;
      }
      phase_transpose(P, R, false, smem);
      if (!grid_sync(P)) return;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched Pauli-frame sampling (Sec. 5, Alg. 9) of the persistent part's
// circuits, one launch for all of them: an item is (circuit, 64-shot word);
// a block runs the circuit's whole program on that word's frame slice held
// in shared memory (X~, Z~ of every qubit, 16 n bytes): frame init from the
// keyed Philox words, every layer's gates without signs (barrier between
// layers), and for each measurement m of qubit q the output X~[q] ^ ref[m]
// followed by Z~[q] <- the keyed word of event m + 1. Frames of different
// shot words never interact, so the items are independent. The words equal
// qs_sim_sample's for the same circuit and seed.
// ---------------------------------------------------------------------------
struct BSampleCirc {
  uint32_t c, nrounds, rtab, ow;  // circuit, rounds, offset of its round table, shot words
  uint64_t shots, seed;
  uint64_t *out;                  // [M][ow] words
};

__global__ void __launch_bounds__(128)
batch_sample_kernel(const BCirc *__restrict__ circs, const BSampleCirc *__restrict__ sc, uint32_t nsc,
                    const uint64_t *__restrict__ pre, const uint32_t *__restrict__ rtab,
                    uint64_t total, uint32_t *__restrict__ err) {
  extern __shared__ uint64_t fr[];  // [2][nmax]
  const uint32_t tid = threadIdx.x;
  for (uint64_t item = blockIdx.x; item < total; item += gridDim.x) {
    uint32_t lo = 0, hi = nsc;  // circuit s with pre[s] <= item < pre[s + 1]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (pre[mid] <= item) lo = mid; else hi = mid;
    }
    const BSampleCirc S = sc[lo];
    const BCirc &C = circs[S.c];
    const uint32_t n = C.n;
    const uint64_t j = item - pre[lo];
    uint64_t *FX = fr, *FZ = fr + n;
    for (uint32_t q = tid; q < n; q += blockDim.x) {
      FX[q] = 0;
      FZ[q] = philox4x64_10(0, q, j >> 2, 1, S.seed, kFrameKey).v[j & 3];
    }
    __syncthreads();
    const uint64_t mask = (j == S.ow - 1 && (S.shots & 63)) ? (1ull << (S.shots & 63)) - 1 : ~0ull;
    const uint32_t *rl = rtab + S.rtab, *rm = rl + S.nrounds + 1;
    for (uint32_t r = 0; r < S.nrounds; ++r) {
      for (uint32_t l = rl[r]; l < rl[r + 1]; ++l) {
        const int64_t g1 = C.lptr[l + 1];
        for (int64_t g = C.lptr[l] + tid; g < g1; g += blockDim.x) {
          const uint32_t w = C.gates[2 * g], qb = C.gates[2 * g + 1];
          const uint32_t type = w >> 24, qa = w & 0xFFFFFFu;
          const bool two = type >= QS_CX && type <= QS_ISWAP;
          if (qa >= n || type >= QS_NUM_GATE_TYPES || (two && (qb >= n || qb == qa))) {
            atomicOr(err, kErrBadGate);
            continue;
          }
          uint64_t xa = FX[qa], za = FZ[qa], xb = 0, zb = 0, s = 0;
          if (two) { xb = FX[qb]; zb = FZ[qb]; }
          rule<false>(type, xa, za, xb, zb, s);
          FX[qa] = xa;
          FZ[qa] = za;
          if (two) { FX[qb] = xb; FZ[qb] = zb; }
        }
        __syncthreads();
      }
      // measurements of the round: outputs read X~ only; Z~[q] takes the word
      // of the last measurement of q in the round
      const uint32_t m0 = rm[r], m1 = rm[r + 1];
      for (uint32_t m = m0 + tid; m < m1; m += blockDim.x) {
        const uint32_t q = C.qubits[m];
        const uint64_t ref = C.record[m] ? ~0ull : 0ull;
        S.out[(uint64_t)m * S.ow + j] = (FX[q] ^ ref) & mask;
      }
      __syncthreads();
      for (uint32_t m = m0 + tid; m < m1; m += blockDim.x) {
        const uint32_t q = C.qubits[m];
        bool last = true;
        for (uint32_t m2 = m + 1; m2 < m1; ++m2)
          if (C.qubits[m2] == q) { last = false; break; }
        if (last) FZ[q] = philox4x64_10((uint64_t)m + 1, q, j >> 2, 1, S.seed, kFrameKey).v[j & 3];
      }
      __syncthreads();
    }
  }
}

}  // namespace qs

using namespace qs;

namespace {

thread_local std::string g_batch_err;

int bfail(int code, const std::string &msg) {
  g_batch_err = msg;
  return code;
}

struct Carve2 {
  size_t off = 0;
  size_t take(size_t b) {
    size_t o = off;
    off += (b + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace

// A large circuit of the batch, simulated by its own qs_sim on a worker stream.
struct BSim {
  uint32_t index = 0;
  qs_sim *sim = nullptr;
  uint32_t *packed_dev = nullptr;  // qs_pack_layers records, device
  std::vector<int64_t> lp;         // layer offsets
  std::vector<uint32_t> rl, rm, qubits;
  uint64_t seed = 0, shot = 0;
};

struct qs_batch {
  cudaStream_t stream = nullptr;
  void *ws = nullptr;
  bool owns = false, broken = false;
  uint32_t count = 0, nrounds = 0, n_max = 0;
  std::vector<BCirc> circs;            // host copy, device pointers
  std::vector<uint64_t> meas_total;    // per circuit
  std::vector<std::vector<uint32_t>> rl, rm;  // per circuit round layer / measurement offsets
  BCirc *d_circs = nullptr;
  BAct *d_acts = nullptr;
  BRound *d_rounds = nullptr;
  uint64_t *d_pre_n = nullptr;
  uint32_t *d_bar = nullptr, *d_err = nullptr;
  uint64_t *zero_begin = nullptr;
  uint64_t zero_words = 0;
  size_t acts_cap = 0;
  uint32_t built_wpb = 0;
  uint64_t signature = 0;
  int sms = 152;
  bool any_small = false;               // the persistent kernel has work
  std::vector<int32_t> sim_of;          // per circuit: index into sims, or -1
  std::vector<BSim> sims;
  std::vector<cudaStream_t> wstreams;   // worker streams of the large circuits
  std::vector<cudaEvent_t> wevents;
  cudaEvent_t start_ev = nullptr;       // worker streams start after the batch stream's earlier work
  bool skip_sims = false;               // set while autotuning the persistent kernel
  bool ran_full = false;                // the records are those of a complete qs_batch_run
};

static void free_sims(qs_batch *b) {
  for (BSim &x : b->sims) {
    if (x.sim) qs_sim_destroy(x.sim);
    if (x.packed_dev) cudaFree(x.packed_dev);
  }
  b->sims.clear();
  for (cudaEvent_t e : b->wevents) cudaEventDestroy(e);
  for (cudaStream_t st : b->wstreams) cudaStreamDestroy(st);
  if (b->start_ev) cudaEventDestroy(b->start_ev);
  b->start_ev = nullptr;
  b->wevents.clear();
  b->wstreams.clear();
}

static void layout_of(uint32_t n, uint32_t &k, uint32_t &cs, uint32_t &ncols, uint32_t &rs,
                      uint32_t &nrows) {
  Layout L = make_layout(n);
  k = L.k; cs = L.cs; ncols = L.ncols; rs = L.rs; nrows = (uint32_t)L.nrows;
}

struct BatchPlan {
  std::vector<size_t> off_X, off_Z, off_S, off_RX, off_RZ, off_colx, off_mst, off_dx, off_dz,
      off_ds, off_rec, off_g, off_lp, off_q;
  size_t zero_end = 0, circs = 0, acts = 0, rounds = 0, pre_n = 0, bar = 0, err = 0, total = 0;
  size_t acts_cap = 0;
};

static int plan_batch(uint32_t count, const qs_batch_circuit *cc, BatchPlan &P, uint32_t &nrounds) {
  Carve2 c;
  P.off_X.resize(count); P.off_Z.resize(count); P.off_S.resize(count);
  nrounds = 0;
  size_t acts = 0;
  for (uint32_t i = 0; i < count; ++i) {
    uint32_t k, cs, ncols, rs, nrows;
    layout_of(cc[i].n, k, cs, ncols, rs, nrows);
    P.off_X[i] = c.take((size_t)ncols * cs * 8);
    P.off_Z[i] = c.take((size_t)ncols * cs * 8);
    P.off_S[i] = c.take((size_t)cs * 8);
    nrounds = std::max(nrounds, cc[i].n_rounds);
    acts += 2 * (size_t)cc[i].n_rounds;
  }
  P.zero_end = c.off;
  P.off_RX.resize(count); P.off_RZ.resize(count); P.off_colx.resize(count); P.off_mst.resize(count);
  P.off_dx.resize(count); P.off_dz.resize(count); P.off_ds.resize(count); P.off_rec.resize(count);
  P.off_g.resize(count); P.off_lp.resize(count); P.off_q.resize(count);
  for (uint32_t i = 0; i < count; ++i) {
    uint32_t k, cs, ncols, rs, nrows;
    layout_of(cc[i].n, k, cs, ncols, rs, nrows);
    P.off_RX[i] = c.take((size_t)nrows * rs * 8);
    P.off_RZ[i] = c.take((size_t)nrows * rs * 8);
    P.off_colx[i] = c.take((size_t)cs * 8);
    P.off_mst[i] = c.take(kMeasStateWords * 8);
    P.off_dx[i] = c.take((size_t)k * rs * 8);
    P.off_dz[i] = c.take((size_t)k * rs * 8);
    P.off_ds[i] = c.take((size_t)k * 4);
    const uint32_t nrr = cc[i].n_rounds;
    const uint64_t M = nrr ? cc[i].round_meas[nrr] : 0;
    P.off_rec[i] = c.take(std::max<uint64_t>(M, 1));
    const int64_t G = cc[i].n_layers ? cc[i].layer_ptr[cc[i].n_layers] : 0;
    P.off_g[i] = c.take((size_t)std::max<int64_t>(G, 1) * 8);
    P.off_lp[i] = c.take(((size_t)cc[i].n_layers + 1) * 8);
    P.off_q[i] = c.take((size_t)std::max<uint64_t>(M, 1) * 4);
  }
  P.acts_cap = acts + 2 * (size_t)nrounds + 2;
  P.circs = c.take(count * sizeof(BCirc));
  P.acts = c.take(P.acts_cap * sizeof(BAct));
  P.rounds = c.take((size_t)std::max<uint32_t>(nrounds, 1) * sizeof(BRound));
  P.pre_n = c.take(((size_t)count + 1) * 8);
  P.bar = c.take(64);
  P.err = c.take(64);
  P.total = c.off;
  return QS_OK;
}

static int validate_batch(uint32_t count, const qs_batch_circuit *cc) {
  if (count == 0 || !cc) return bfail(QS_ERR_ARG, "empty batch");
  char buf[200];
  for (uint32_t i = 0; i < count; ++i) {
    const qs_batch_circuit &c = cc[i];
    if (c.n == 0 || c.n > kBatchLimitQubits) {
      snprintf(buf, sizeof buf, "circuit %u: n must be in [1, %u]", i, kBatchLimitQubits);
      return bfail(QS_ERR_ARG, buf);
    }
    if (c.n_layers && (!c.layer_ptr || (!c.gates && c.layer_ptr[c.n_layers] > 0)))
      return bfail(QS_ERR_ARG, "NULL gates or layer_ptr");
    if (c.n_rounds && (!c.round_layers || !c.round_meas))
      return bfail(QS_ERR_ARG, "NULL round arrays");
    for (uint32_t r = 0; r < c.n_rounds; ++r) {
      if (c.round_layers[r] > c.round_layers[r + 1] || c.round_layers[r + 1] > c.n_layers ||
          c.round_meas[r] > c.round_meas[r + 1]) {
        snprintf(buf, sizeof buf, "circuit %u round %u: offsets must be nondecreasing and in range",
                 i, r);
        return bfail(QS_ERR_ARG, buf);
      }
    }
    if (c.n_rounds && c.round_layers[0] != 0) return bfail(QS_ERR_ARG, "round_layers[0] must be 0");
    if (c.n_rounds && c.round_meas[0] != 0) return bfail(QS_ERR_ARG, "round_meas[0] must be 0");
    const uint64_t M = c.n_rounds ? c.round_meas[c.n_rounds] : 0;
    if (M && !c.qubits) return bfail(QS_ERR_ARG, "NULL qubits");
    for (uint64_t m = 0; m < M; ++m)
      if (c.qubits[m] >= c.n) {
        snprintf(buf, sizeof buf, "circuit %u: measured qubit out of range", i);
        return bfail(QS_ERR_ARG, buf);
      }
  }
  return QS_OK;
}

// Builds the per-round work lists for a gate-phase slice width `wpb`.
static int build_acts(qs_batch *b, uint32_t wpb) {
  std::vector<BAct> acts;
  std::vector<BRound> rounds(std::max<uint32_t>(b->nrounds, 1));
  std::vector<uint64_t> m0(b->count, 0);
  for (uint32_t r = 0; r < b->nrounds; ++r) {
    BRound R{};
    R.g_first = (uint32_t)acts.size();
    uint64_t pre = 0;
    for (uint32_t c = 0; c < b->count; ++c) {
      if (r >= b->rl[c].size() - 1) continue;
      const uint32_t l0 = b->rl[c][r], l1 = b->rl[c][r + 1];
      if (l1 <= l0) continue;
      BAct a{};
      a.c = c; a.l0 = l0; a.l1 = l1; a.pre = pre;
      acts.push_back(a);
      pre += (b->circs[c].cs + wpb - 1) / wpb;
    }
    R.g_count = (uint32_t)acts.size() - R.g_first;
    { BAct s{}; s.pre = pre; acts.push_back(s); }
    // measurement list, sorted by count (descending), then circuit
    std::vector<uint32_t> mc;
    for (uint32_t c = 0; c < b->count; ++c) {
      if (r >= b->rm[c].size() - 1) continue;
      if (b->rm[c][r + 1] > b->rm[c][r]) mc.push_back(c);
    }
    std::stable_sort(mc.begin(), mc.end(), [&](uint32_t x, uint32_t y) {
      return (b->rm[x][r + 1] - b->rm[x][r]) > (b->rm[y][r + 1] - b->rm[y][r]);
    });
    R.m_first = (uint32_t)acts.size();
    uint64_t pt = 0, pr = 0, pu = 0;
    R.max_qn = 0;
    for (uint32_t c : mc) {
      BAct a{};
      a.c = c; a.q0 = b->rm[c][r]; a.qn = b->rm[c][r + 1] - b->rm[c][r];
      a.m0 = a.q0;
      a.pre = pt; a.pre2 = pr; a.pre3 = pu;
      acts.push_back(a);
      const BCirc &C = b->circs[c];
      pt += 2ull * (C.cs / 4) * (C.ncols / 256);
      pr += C.nrows;
      pu += C.nrows / (32 / C.lpr);
      R.max_qn = std::max(R.max_qn, a.qn);
    }
    R.m_count = (uint32_t)mc.size();
    { BAct s{}; s.pre = pt; s.pre2 = pr; s.pre3 = pu; acts.push_back(s); }
    rounds[r] = R;
  }
  if (acts.size() > b->acts_cap) return bfail(QS_ERR_INTERNAL, "work list capacity");
  cudaError_t e = cudaMemcpyAsync(b->d_acts, acts.data(), acts.size() * sizeof(BAct),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_rounds, rounds.data(), rounds.size() * sizeof(BRound),
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->broken = true;
    return bfail(QS_ERR_CUDA, std::string("upload of work lists: ") + cudaGetErrorString(e));
  }
  b->built_wpb = wpb;
  return QS_OK;
}

// The persistent kernel's view of the batch: large circuits become empty
// one-qubit programs (their work runs through per-circuit simulators).
static std::vector<qs_batch_circuit> kernel_view(uint32_t count, const qs_batch_circuit *cc) {
  std::vector<qs_batch_circuit> v(cc, cc + count);
  for (qs_batch_circuit &c : v)
    if (c.n >= kBatchSimMinQubits) {
      const uint64_t seed = c.seed, shot = c.shot;
      c = qs_batch_circuit{};
      c.n = 1;
      c.seed = seed;
      c.shot = shot;
    }
  return v;
}

extern "C" {

const char *qs_batch_last_error(void) { return g_batch_err.c_str(); }

size_t qs_batch_required_bytes(uint32_t count, const qs_batch_circuit *circuits) {
  if (validate_batch(count, circuits)) return 0;
  const std::vector<qs_batch_circuit> kv = kernel_view(count, circuits);
  BatchPlan P;
  uint32_t nr;
  plan_batch(count, kv.data(), P, nr);
  return P.total;
}

int qs_batch_create(uint32_t count, const qs_batch_circuit *cc, void *stream, void *workspace,
                    size_t workspace_bytes, qs_batch **out) {
  if (!out) return bfail(QS_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate_batch(count, cc);
  if (rc) return rc;
  const qs_batch_circuit *orig = cc;
  const std::vector<qs_batch_circuit> kv = kernel_view(count, cc);
  cc = kv.data();
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255))
    return bfail(QS_ERR_ARG, "workspace must be 256-byte aligned");
  BatchPlan P;
  qs_batch *b = new (std::nothrow) qs_batch();
  if (!b) return bfail(QS_ERR_OOM, "host allocation failed");
  plan_batch(count, cc, P, b->nrounds);
  b->stream = static_cast<cudaStream_t>(stream);
  b->count = count;
  if (workspace) {
    if (workspace_bytes < P.total) { delete b; return bfail(QS_ERR_SIZE, "workspace too small"); }
    b->ws = workspace;
  } else {
    if (cudaMalloc(&b->ws, P.total) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return bfail(QS_ERR_OOM, "cudaMalloc of the batch failed");
    }
    b->owns = true;
  }
  uint8_t *base = static_cast<uint8_t *>(b->ws);
  b->circs.resize(count);
  b->meas_total.resize(count);
  b->rl.resize(count);
  b->rm.resize(count);
  std::vector<uint64_t> pre_n(count + 1, 0);
  uint64_t sig = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { sig = (sig ^ v) * 1099511628211ull; };
  mix(count);
  cudaError_t e = cudaSuccess;
  for (uint32_t i = 0; i < count && e == cudaSuccess; ++i) {
    const qs_batch_circuit &c = cc[i];
    BCirc C{};
    C.n = c.n;
    layout_of(c.n, C.k, C.cs, C.ncols, C.rs, C.nrows);
    C.lpr = 1;
    while (C.lpr < 32 && C.lpr < C.rs / 2) C.lpr <<= 1;
    C.X = reinterpret_cast<uint64_t *>(base + P.off_X[i]);
    C.Z = reinterpret_cast<uint64_t *>(base + P.off_Z[i]);
    C.S = reinterpret_cast<uint64_t *>(base + P.off_S[i]);
    C.RX = reinterpret_cast<uint64_t *>(base + P.off_RX[i]);
    C.RZ = reinterpret_cast<uint64_t *>(base + P.off_RZ[i]);
    C.colx = reinterpret_cast<uint32_t *>(base + P.off_colx[i]);
    C.mst = reinterpret_cast<int64_t *>(base + P.off_mst[i]);
    C.det_x = reinterpret_cast<uint64_t *>(base + P.off_dx[i]);
    C.det_z = reinterpret_cast<uint64_t *>(base + P.off_dz[i]);
    C.det_scal = reinterpret_cast<int32_t *>(base + P.off_ds[i]);
    C.record = base + P.off_rec[i];
    C.seed = c.seed;
    C.shot = c.shot;
    const int64_t G = c.n_layers ? c.layer_ptr[c.n_layers] : 0;
    std::vector<uint32_t> packed(2 * (size_t)std::max<int64_t>(G, 1), 0);
    std::vector<int64_t> lp(c.n_layers + 1, 0);
    if (c.n_layers) {
      rc = qs_pack_layers(c.n, c.gates, c.layer_ptr, c.n_layers, packed.data());
      if (rc) {
        g_batch_err = std::string("circuit ") + std::to_string(i) + ": " + qs_last_error();
        if (b->owns) cudaFree(b->ws);
        delete b;
        return rc;
      }
      lp.assign(c.layer_ptr, c.layer_ptr + c.n_layers + 1);
    }
    C.gates = reinterpret_cast<const uint32_t *>(base + P.off_g[i]);
    C.lptr = reinterpret_cast<const int64_t *>(base + P.off_lp[i]);
    C.qubits = reinterpret_cast<const uint32_t *>(base + P.off_q[i]);
    const uint64_t M = c.n_rounds ? c.round_meas[c.n_rounds] : 0;
    e = cudaMemcpy(base + P.off_g[i], packed.data(), packed.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(base + P.off_lp[i], lp.data(), lp.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && M)
      e = cudaMemcpy(base + P.off_q[i], c.qubits, M * 4, cudaMemcpyHostToDevice);
    b->circs[i] = C;
    b->meas_total[i] = M;
    b->rl[i].assign(c.round_layers ? c.round_layers : nullptr,
                    c.round_layers ? c.round_layers + c.n_rounds + 1 : nullptr);
    b->rm[i].assign(c.round_meas ? c.round_meas : nullptr,
                    c.round_meas ? c.round_meas + c.n_rounds + 1 : nullptr);
    if (b->rl[i].empty()) { b->rl[i].push_back(0); b->rm[i].push_back(0); }
    if (orig[i].n < kBatchSimMinQubits && (G > 0 || M > 0)) b->any_small = true;
    pre_n[i + 1] = pre_n[i] + c.n;
    b->n_max = std::max(b->n_max, c.n);
    mix(c.n); mix(c.n_rounds); mix((uint64_t)G); mix(M);
  }
  b->signature = sig;
  b->d_circs = reinterpret_cast<BCirc *>(base + P.circs);
  b->d_acts = reinterpret_cast<BAct *>(base + P.acts);
  b->d_rounds = reinterpret_cast<BRound *>(base + P.rounds);
  b->d_pre_n = reinterpret_cast<uint64_t *>(base + P.pre_n);
  b->d_bar = reinterpret_cast<uint32_t *>(base + P.bar);
  b->d_err = reinterpret_cast<uint32_t *>(base + P.err);
  b->zero_begin = reinterpret_cast<uint64_t *>(base);
  b->zero_words = P.zero_end / 8;
  b->acts_cap = P.acts_cap;
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_circs, b->circs.data(), count * sizeof(BCirc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_pre_n, pre_n.data(), pre_n.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 64);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    if (b->owns) cudaFree(b->ws);
    delete b;
    return bfail(QS_ERR_CUDA, std::string("batch upload: ") + cudaGetErrorString(e));
  }
  // large circuits: one simulator each, spread over the worker streams by size
  b->sim_of.assign(count, -1);
  std::vector<uint32_t> large;
  for (uint32_t i = 0; i < count; ++i)
    if (orig[i].n >= kBatchSimMinQubits) large.push_back(i);
  std::stable_sort(large.begin(), large.end(),
                   [&](uint32_t x, uint32_t y) { return orig[x].n > orig[y].n; });
  const uint32_t nw = std::min<uint32_t>(kBatchMaxWorkers, (uint32_t)large.size());
  if (nw && cudaEventCreateWithFlags(&b->start_ev, cudaEventDisableTiming) != cudaSuccess)
    rc = bfail(QS_ERR_CUDA, "batch event creation failed");
  for (uint32_t w = 0; w < nw && rc == QS_OK; ++w) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      rc = bfail(QS_ERR_CUDA, "worker stream creation failed");
      break;
    }
    b->wstreams.push_back(st);
    b->wevents.push_back(ev);
  }
  for (size_t j = 0; j < large.size() && rc == QS_OK; ++j) {
    const uint32_t i = large[j];
    const qs_batch_circuit &c = orig[i];
    BSim x;
    x.index = i;
    x.seed = c.seed;
    x.shot = c.shot;
    const uint64_t M = c.n_rounds ? c.round_meas[c.n_rounds] : 0;
    b->meas_total[i] = M;
    x.rl.assign(c.round_layers ? c.round_layers : nullptr,
                c.round_layers ? c.round_layers + c.n_rounds + 1 : nullptr);
    x.rm.assign(c.round_meas ? c.round_meas : nullptr,
                c.round_meas ? c.round_meas + c.n_rounds + 1 : nullptr);
    if (M) x.qubits.assign(c.qubits, c.qubits + M);
    const int64_t G = c.n_layers ? c.layer_ptr[c.n_layers] : 0;
    x.lp.assign(c.layer_ptr ? c.layer_ptr : nullptr, c.layer_ptr ? c.layer_ptr + c.n_layers + 1 : nullptr);
    if (x.lp.empty()) x.lp.push_back(0);
    std::vector<uint32_t> packed(2 * (size_t)std::max<int64_t>(G, 1), 0);
    if (c.n_layers && (rc = qs_pack_layers(c.n, c.gates, c.layer_ptr, c.n_layers, packed.data()))) {
      rc = bfail(rc, std::string("circuit ") + std::to_string(i) + ": " + qs_last_error());
      break;
    }
    if (cudaMalloc(&x.packed_dev, packed.size() * 4) != cudaSuccess ||
        cudaMemcpy(x.packed_dev, packed.data(), packed.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      if (x.packed_dev) cudaFree(x.packed_dev);
      rc = bfail(QS_ERR_OOM, "gate records of a large circuit");
      break;
    }
    qs_options opt{};
    opt.record_capacity = std::max<uint64_t>(M, 1);
    if ((rc = qs_sim_create(c.n, &opt, b->wstreams[j % nw], nullptr, 0, &x.sim))) {
      cudaFree(x.packed_dev);
      rc = bfail(rc, std::string("circuit ") + std::to_string(i) + ": " + qs_last_error());
      break;
    }
    b->sim_of[i] = (int32_t)b->sims.size();
    b->sims.push_back(std::move(x));
  }
  if (rc != QS_OK) {
    free_sims(b);
    if (b->owns) cudaFree(b->ws);
    delete b;
    return rc;
  }
  *out = b;
  return QS_OK;
}

int qs_batch_destroy(qs_batch *b) {
  if (!b) return QS_OK;
  cudaStreamSynchronize(b->stream);
  free_sims(b);
  if (b->owns && b->ws) cudaFree(b->ws);
  delete b;
  return QS_OK;
}

static int tuning_ok(const qs_batch *b, const qs_batch_tuning &t, size_t *smem) {
  if (t.threads != 256 && t.threads != 512 && t.threads != 1024)
    return bfail(QS_ERR_ARG, "tuning.threads must be 256, 512 or 1024");
  if (t.words_per_block != 1 && t.words_per_block != 2)
    return bfail(QS_ERR_ARG, "tuning.words_per_block must be 1 or 2");
  const size_t gate_smem = (size_t)16 * b->n_max * t.words_per_block;
  const size_t tile_smem = (size_t)(t.threads / 128) * 256 * 5 * 8;
  *smem = std::max(gate_smem, tile_smem);
  if (*smem > 227 * 1024) return bfail(QS_ERR_ARG, "tuning needs more than 227 KB of shared memory");
  return QS_OK;
}

static int run_kernel(qs_batch *b, const qs_batch_tuning *tuning, uint32_t round_limit);
static int batch_run(qs_batch *b, const qs_batch_tuning *tuning, uint32_t round_limit);

// Enqueues every large circuit's rounds on its simulator, one host thread per
// worker stream (blocked measurement waits for its stream once per block),
// then makes the batch stream wait for the worker streams.
static int run_sims(qs_batch *b, uint32_t round_limit) {
  const uint32_t nw = (uint32_t)b->wstreams.size();
  std::mutex mu;
  int first_rc = QS_OK;
  std::string first_msg;
  auto worker = [&](uint32_t w) {
    int rc = QS_OK;
    if (cudaStreamWaitEvent(b->wstreams[w], b->start_ev, 0) != cudaSuccess) rc = QS_ERR_CUDA;
    for (size_t j = w; j < b->sims.size() && rc == QS_OK; j += nw) {
      BSim &x = b->sims[j];
      rc = qs_sim_reset(x.sim, nullptr);
      const uint32_t nr = x.rl.empty() ? 0 : (uint32_t)x.rl.size() - 1;
      const uint32_t lim = std::min(nr, round_limit);
      for (uint32_t r = 0; r < lim && rc == QS_OK; ++r) {
        if (x.rl[r + 1] > x.rl[r])
          rc = qs_sim_apply_layers_dev(x.sim, x.packed_dev, x.lp.data(), x.rl[r], x.rl[r + 1]);
        if (rc == QS_OK && x.rm[r + 1] > x.rm[r])
          rc = qs_sim_measure(x.sim, x.qubits.data() + x.rm[r], x.rm[r + 1] - x.rm[r],
                              qs_key{x.seed, x.shot}, nullptr);
      }
      if (rc != QS_OK) {
        std::lock_guard<std::mutex> lock(mu);
        if (first_rc == QS_OK) {
          first_rc = rc;
          first_msg = std::string("circuit ") + std::to_string(x.index) + ": " + qs_last_error();
        }
      }
    }
    if (cudaEventRecord(b->wevents[w], b->wstreams[w]) != cudaSuccess) {
      std::lock_guard<std::mutex> lock(mu);
      if (first_rc == QS_OK) { first_rc = QS_ERR_CUDA; first_msg = "worker event record failed"; }
    }
  };
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::thread> threads;
  for (uint32_t w = 0; w < nw; ++w)
    threads.emplace_back([&, w]() {
      cudaSetDevice(dev);
      worker(w);
    });
  for (std::thread &t : threads) t.join();
  for (uint32_t w = 0; w < nw && first_rc == QS_OK; ++w)
    if (cudaStreamWaitEvent(b->stream, b->wevents[w], 0) != cudaSuccess) {
      first_rc = QS_ERR_CUDA;
      first_msg = "batch stream wait failed";
    }
  if (first_rc != QS_OK) return bfail(first_rc, first_msg);
  return QS_OK;
}

int qs_batch_run(qs_batch *b, const qs_batch_tuning *tuning, uint32_t round_limit) {
  nvtxRangePushA("qs_batch_run");
  const int rc = batch_run(b, tuning, round_limit);
  nvtxRangePop();
  return rc;
}

static int batch_run(qs_batch *b, const qs_batch_tuning *tuning, uint32_t round_limit) {
  if (!b) return bfail(QS_ERR_ARG, "batch is NULL");
  if (b->broken) return bfail(QS_ERR_STATE, "batch is unusable after an earlier device error");
  b->ran_full = (round_limit == 0 || round_limit >= b->nrounds) && !b->skip_sims;
  int rc = QS_OK;
  const bool sims = !b->skip_sims && !b->sims.empty();
  if (sims && cudaEventRecord(b->start_ev, b->stream) != cudaSuccess)
    return bfail(QS_ERR_CUDA, "batch event record failed");
  if (b->any_small || b->sims.empty()) {
    if ((rc = run_kernel(b, tuning, round_limit))) return rc;
  }
  if (sims) rc = run_sims(b, round_limit ? round_limit : 0xFFFFFFFFu);
  return rc;
}

static int run_kernel(qs_batch *b, const qs_batch_tuning *tuning, uint32_t round_limit) {
  qs_batch_tuning t = tuning ? *tuning : qs_batch_tuning{512, 0, 1, 0, 0};
  if (t.spin_limit == 0) t.spin_limit = 20ull * 1000 * 1000;  // x >=128 ns: several seconds
  size_t smem = 0;
  int rc = tuning_ok(b, t, &smem);
  if (rc) return rc;
  if (b->built_wpb != t.words_per_block && (rc = build_acts(b, t.words_per_block))) return rc;
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, (int)t.threads, smem);
  if (e != cudaSuccess || per_sm < 1) {
    return bfail(QS_ERR_ARG, std::string("batch kernel does not fit with this tuning: ") +
                                 cudaGetErrorString(e));
  }
  if (t.blocks_per_sm) per_sm = std::min<int>(per_sm, (int)t.blocks_per_sm);
  BProg P;
  P.circs = b->d_circs;
  P.acts = b->d_acts;
  P.rounds = b->d_rounds;
  P.pre_n = b->d_pre_n;
  P.zero_begin = b->zero_begin;
  P.zero_words = b->zero_words;
  P.spin_limit = t.spin_limit;
  P.ncirc = b->count;
  P.nrounds = b->nrounds;
  P.wpb = t.words_per_block;
  P.fuse_depth = t.fuse_depth;
  P.bar = b->d_bar;
  P.err = b->d_err;
  uint32_t rl = round_limit ? round_limit : 0xFFFFFFFFu;
  e = cudaMemsetAsync(b->d_bar, 0, 64, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 64, b->stream);
  if (e == cudaSuccess) {
    void *args[] = {&P, &rl};
    e = cudaLaunchCooperativeKernel((void *)batch_kernel, dim3(per_sm * b->sms), dim3(t.threads),
                                    args, smem, b->stream);
  }
  if (e != cudaSuccess) {
    b->broken = true;
    return bfail(QS_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  }
  return QS_OK;
}

int qs_batch_sync(qs_batch *b) {
  if (!b) return bfail(QS_ERR_ARG, "batch is NULL");
  if (b->broken) return bfail(QS_ERR_STATE, "batch is unusable after an earlier device error");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  uint32_t flags = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flags, b->d_err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    b->broken = true;
    return bfail(QS_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(e));
  }
  if (flags & kErrTimeout) return bfail(QS_ERR_TIMEOUT, "a grid barrier of the batch kernel ran out");
  if (flags) {
    char buf[96];
    snprintf(buf, sizeof buf, "batch self-check failed (flags 0x%x)", flags);
    return bfail(QS_ERR_INTERNAL, buf);
  }
  for (BSim &x : b->sims) {
    const int rc = qs_sim_sync(x.sim);
    if (rc) return bfail(rc, std::string("circuit ") + std::to_string(x.index) + ": " + qs_last_error());
  }
  return QS_OK;
}

int qs_batch_record(qs_batch *b, uint32_t circuit, uint8_t *dst, size_t count) {
  if (!b || circuit >= b->count) return bfail(QS_ERR_ARG, "bad batch or circuit index");
  if (count > b->meas_total[circuit]) return bfail(QS_ERR_ARG, "count beyond the circuit's record");
  if (count && !dst) return bfail(QS_ERR_ARG, "dst is NULL");
  int rc = qs_batch_sync(b);
  if (rc) return rc;
  if (b->sim_of[circuit] >= 0) {
    rc = count ? qs_sim_record(b->sims[b->sim_of[circuit]].sim, 0, count, dst) : QS_OK;
    return rc ? bfail(rc, qs_last_error()) : QS_OK;
  }
  if (count && cudaMemcpy(dst, b->circs[circuit].record, count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(QS_ERR_CUDA, "record copy failed");
  return QS_OK;
}

int qs_batch_export_rows(qs_batch *b, uint32_t circuit, const uint32_t *rows, uint32_t count,
                         uint64_t *dst) {
  if (!b || circuit >= b->count) return bfail(QS_ERR_ARG, "bad batch or circuit index");
  int rc = qs_batch_sync(b);
  if (rc) return rc;
  if (b->sim_of[circuit] >= 0) {
    rc = qs_sim_export_rows(b->sims[b->sim_of[circuit]].sim, rows, count, dst);
    return rc ? bfail(rc, qs_last_error()) : QS_OK;
  }
  const BCirc &C = b->circs[circuit];
  for (uint32_t i = 0; i < count; ++i)
    if (rows[i] >= 2 * C.n) return bfail(QS_ERR_ARG, "row index >= 2n");
  // the column-major tableau is current after a run; rebuild the row-major copy
  Dev d{};
  d.L = make_layout(C.n);
  d.X = C.X; d.Z = C.Z; d.RX = C.RX; d.RZ = C.RZ;
  d.err = b->d_err;
  cudaError_t e = launch_to_rows(d, b->stream);
  std::vector<uint64_t> S(C.cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S.data(), C.S, (size_t)C.cs * 8, cudaMemcpyDeviceToHost, b->stream);
  const size_t per = 2ull * C.k + 1;
  for (uint32_t i = 0; i < count && e == cudaSuccess; ++i) {
    const uint64_t pr = rows[i] < C.n ? rows[i] : 64ull * C.k + (rows[i] - C.n);
    e = cudaMemcpyAsync(dst + i * per, C.RX + pr * C.rs, (size_t)C.k * 8, cudaMemcpyDeviceToHost,
                        b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst + i * per + C.k, C.RZ + pr * C.rs, (size_t)C.k * 8,
                          cudaMemcpyDeviceToHost, b->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->broken = true;
    return bfail(QS_ERR_CUDA, std::string("batch export: ") + cudaGetErrorString(e));
  }
  for (uint32_t i = 0; i < count; ++i) {
    const uint64_t pr = rows[i] < C.n ? rows[i] : 64ull * C.k + (rows[i] - C.n);
    dst[i * per + 2 * C.k] = (S[pr >> 6] >> (pr & 63)) & 1u;
  }
  return QS_OK;
}

int qs_batch_autotune(qs_batch *b, uint32_t round_limit, const char *cache_path,
                      qs_batch_tuning *best) {
  if (!b || !best) return bfail(QS_ERR_ARG, "NULL argument");
  char dev_name[256] = "gpu";
  {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
      snprintf(dev_name, sizeof dev_name, "%s", prop.name);
  }
  char key[400];
  snprintf(key, sizeof key, "%s|%016llx|%u", dev_name, (unsigned long long)b->signature, round_limit);
  for (char *p = key; *p; ++p)
    if (*p == ' ') *p = '_';
  if (cache_path) {
    std::ifstream f(cache_path);
    std::string line;
    while (std::getline(f, line)) {
      std::istringstream ss(line);
      std::string k2;
      qs_batch_tuning t{};
      if (ss >> k2 >> t.threads >> t.blocks_per_sm >> t.words_per_block >> t.fuse_depth && k2 == key) {
        size_t smem;
        if (tuning_ok(b, t, &smem) == QS_OK) {
          *best = t;
          return QS_OK;
        }
      }
    }
  }
  if (!b->any_small) {  // every circuit runs through a simulator: nothing to tune
    *best = qs_batch_tuning{512, 0, 1, 0, 0};
    return QS_OK;
  }
  b->skip_sims = true;  // time the persistent kernel alone
  const uint32_t threads[] = {256, 512, 1024};
  const uint32_t bps[] = {1, 2, 4};
  const uint32_t wpbs[] = {1, 2};
  const uint32_t depths[] = {0, 1};
  float best_ms = 1e30f;
  qs_batch_tuning best_t{512, 0, 1, 0, 0};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (uint32_t th : threads)
    for (uint32_t bp : bps)
      for (uint32_t w : wpbs)
        for (uint32_t dp : depths) {
          qs_batch_tuning t{th, bp, w, dp, 0};
          size_t smem;
          if (tuning_ok(b, t, &smem) != QS_OK) continue;
          if (th * bp > 2048) continue;
          float ms_min = 1e30f;
          for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, b->stream);
            if (qs_batch_run(b, &t, round_limit) != QS_OK) break;
            cudaEventRecord(e1, b->stream);
            if (qs_batch_sync(b) != QS_OK) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_min = std::min(ms_min, ms);
          }
          if (ms_min < best_ms) { best_ms = ms_min; best_t = t; }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->skip_sims = false;
  g_batch_err.clear();
  *best = best_t;
  if (cache_path && best_ms < 1e29f) {
    std::ofstream f(cache_path, std::ios::app);
    f << key << " " << best_t.threads << " " << best_t.blocks_per_sm << " " << best_t.words_per_block
      << " " << best_t.fuse_depth << "\n";
  }
  return best_ms < 1e29f ? QS_OK : bfail(QS_ERR_INTERNAL, "no tuning candidate ran");
}

int qs_batch_sample(qs_batch *b, const uint64_t *shots, const uint64_t *seeds, uint64_t *const *records) {
  if (!b) return bfail(QS_ERR_ARG, "batch is NULL");
  if (b->broken) return bfail(QS_ERR_STATE, "batch is unusable after an earlier device error");
  if (!shots || !seeds || !records) return bfail(QS_ERR_ARG, "NULL argument");
  if (!b->ran_full) return bfail(QS_ERR_STATE, "sampling needs the records of a complete qs_batch_run");
  // small circuits: one launch; a table of the sampled circuits, their round
  // tables and the prefix of their shot words
  std::vector<BSampleCirc> sc;
  std::vector<uint64_t> pre(1, 0);
  std::vector<uint32_t> rt;
  uint32_t nmax = 1;
  for (uint32_t c = 0; c < b->count; ++c) {
    if (shots[c] == 0) continue;
    if (shots[c] > 2000000000ull) return bfail(QS_ERR_ARG, "shots must be at most 2e9");
    if (!records[c] && b->meas_total[c]) return bfail(QS_ERR_ARG, "records[c] is NULL");
    if (b->sim_of[c] >= 0 || b->meas_total[c] == 0) continue;  // large, or nothing to record
    BSampleCirc x{};
    x.c = c;
    x.nrounds = (uint32_t)b->rl[c].size() - 1;
    x.rtab = (uint32_t)rt.size();
    x.ow = (uint32_t)((shots[c] + 63) / 64);
    x.shots = shots[c];
    x.seed = seeds[c];
    x.out = records[c];
    rt.insert(rt.end(), b->rl[c].begin(), b->rl[c].end());
    rt.insert(rt.end(), b->rm[c].begin(), b->rm[c].end());
    sc.push_back(x);
    pre.push_back(pre.back() + x.ow);
    nmax = std::max(nmax, b->circs[c].n);
  }
  if (!sc.empty()) {
    const size_t bytes_sc = sc.size() * sizeof(BSampleCirc), bytes_pre = pre.size() * 8,
                 bytes_rt = rt.size() * 4;
    const size_t off_pre = (bytes_sc + 255) & ~size_t(255), off_rt = off_pre + ((bytes_pre + 255) & ~size_t(255));
    std::vector<uint8_t> host(off_rt + bytes_rt);
    memcpy(host.data(), sc.data(), bytes_sc);
    memcpy(host.data() + off_pre, pre.data(), bytes_pre);
    memcpy(host.data() + off_rt, rt.data(), bytes_rt);
    void *dev = nullptr;
    cudaError_t e = cudaMallocAsync(&dev, host.size(), b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
      uint8_t *d = static_cast<uint8_t *>(dev);
      const uint64_t total = pre.back();
      const uint32_t grid = (uint32_t)std::min<uint64_t>(total, (uint64_t)b->sms * 16);
      batch_sample_kernel<<<grid, 128, (size_t)2 * nmax * 8, b->stream>>>(
          b->d_circs, reinterpret_cast<const BSampleCirc *>(d), (uint32_t)sc.size(),
          reinterpret_cast<const uint64_t *>(d + off_pre), reinterpret_cast<const uint32_t *>(d + off_rt),
          total, b->d_err);
      e = cudaGetLastError();
      // the host table must outlive the copy: wait for it before returning
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (cudaFreeAsync(dev, b->stream) != cudaSuccess) cudaGetLastError();
    }
    if (e != cudaSuccess) {
      b->broken = true;
      return bfail(QS_ERR_CUDA, std::string("batch sampling: ") + cudaGetErrorString(e));
    }
  }
  // large circuits: their own simulators replay their op logs on the worker streams
  bool any_large = false;
  for (uint32_t c = 0; c < b->count; ++c) any_large |= shots[c] > 0 && b->sim_of[c] >= 0;
  if (any_large) {
    if (cudaEventRecord(b->start_ev, b->stream) != cudaSuccess)
      return bfail(QS_ERR_CUDA, "batch event record failed");
    const uint32_t nw = (uint32_t)b->wstreams.size();
    for (uint32_t w = 0; w < nw; ++w)
      if (cudaStreamWaitEvent(b->wstreams[w], b->start_ev, 0) != cudaSuccess)
        return bfail(QS_ERR_CUDA, "worker stream wait failed");
    for (uint32_t c = 0; c < b->count; ++c) {
      if (!(shots[c] > 0 && b->sim_of[c] >= 0)) continue;
      BSim &x = b->sims[b->sim_of[c]];
      const uint64_t ow = (shots[c] + 63) / 64;
      const int rc = qs_sim_sample(x.sim, shots[c], seeds[c], records[c], b->meas_total[c] * ow, nullptr, 0);
      if (rc) return bfail(rc, std::string("circuit ") + std::to_string(c) + ": " + qs_last_error());
    }
    for (uint32_t w = 0; w < nw; ++w)
      if (cudaEventRecord(b->wevents[w], b->wstreams[w]) != cudaSuccess ||
          cudaStreamWaitEvent(b->stream, b->wevents[w], 0) != cudaSuccess)
        return bfail(QS_ERR_CUDA, "batch stream wait failed");
  }
  return QS_OK;
}

}  // extern "C"
