// Inverse-tableau mode: the paper's measurement variant (Sec. 3.2, Alg. 1 --
// Stim's elimination by CX injection) on the representation it belongs to.
//
// For the Clifford C that prepares the state from |0...0>, the mode keeps the
// images C^dag Z_q C and C^dag X_q C with qubit-indexed signs (Alg. 1's S_S
// and S_D; reading G2 of the paper's sign vectors). Their bits are the
// extended tableau's bits read by columns, so the tableau arrays and both
// layouts are shared with the forward (CHP) mode:
//   image(Z_q): x part at input i = XS[i][q] (stabilizer row i, X column q),
//               z part at input i = XD[i][q] (destabilizer row i), sign SS[q];
//   image(X_q): x part ZS[i][q], z part ZD[i][q], sign SD[q].
// SS and SD are bit vectors of rs words each (bit q % 64 of word q / 64).
//
// Gate layers (Sec. 4.4 Alg. 3 with these signs): a gate G appended to the
// circuit maps each image to that of G^dag P G. The bits follow the column
// rules of Eq. 4; the signs of the gate's qubits follow from the phase of a
// product of two images, a popcount reduction over the n input positions:
//   image(A) image(B) = i^e sigma(sum), e = |xA&zA| + |xB&zB| + 2|zA&xB| - |x'&z'|.
// One block per gate walks the gate's columns (destabilizer word w with the
// stabilizer word k + w: the same input positions), reduces the phases in
// shared memory, and thread 0 updates the sign bits with XOR atomics (gates
// of a layer act on distinct qubits, which may share a sign word).
//
// Measurement (Alg. 1), four launches on the row-major tableau:
//  1. gather (shared with the CHP path): pivot p = smallest stabilizer with
//     XS[p][q] = 1, and the column bits of every row.
//  2. inv_targets: CX injections from the pivot into every later stabilizer t
//     with XS[t][q] = 1 (Alg. 1's GE). The bits are independent per target:
//     S_t ^= S_p. The signs carry the pivot's destabilizer word through the
//     targets in order (Eqs. 9-10); unfolded (Eq. 11), per word u,
//       S ^= sum_k a d_k (1 + zc0 + s_k)  +  a * sum_k d_k E_k,
//     a = pivot stabilizer word, d_k, s_k = target k's destabilizer and old
//     stabilizer words, zc0 = the pivot's destabilizer word, E_k = XOR of d_l
//     over earlier targets. The pair sum is GF(2)-bilinear, so chunks of rows
//     in index order yield independent partials (their XOR D_c, local pair
//     sum L_c, local F_c) -- the paper's three-pass prefix-XOR (Alg. 7) as a
//     chunked scan without a device-wide scan pass.
//  3. inv_combine, per word: the chunks in order give the global pair sum
//     (L_c + Pre_c D_c), the pivot's new destabilizer (zc0 + sum of d) and the
//     sign updates of S_S (x side) and S_D (z side).
//  4. inv_finalize, one block: the H or H_YZ injection on the pivot (by the
//     pivot's destabilizer bit at q), then the X injection when S_S[q]
//     differs from the keyed coin; the outcome is the coin. A deterministic
//     outcome is S_S[q] (nothing changes). Record, kind, pivot reset.
#include <climits>

#include <algorithm>

#include "qs_internal.cuh"

namespace qs {

constexpr int64_t kInvNoPivot = LLONG_MAX;

// ---------------------------------------------------------------------------
// gate layers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool inv_two(uint32_t t) { return t >= QS_CX && t <= QS_ISWAP; }

// phase exponent (mod 4 after summation) of image(A) * image(B) over one
// word of input positions
__device__ __forceinline__ int pprod(uint64_t xa, uint64_t za, uint64_t xb, uint64_t zb) {
  return __popcll(xa & za) + __popcll(xb & zb) + 2 * __popcll(za & xb) -
         __popcll((xa ^ xb) & (za ^ zb));
}

// One column's words for one input word: x and z, destabilizer (d) and
// stabilizer (s) halves.
struct Col { uint64_t xd, xs, zd, zs; };

// bits of the elementary steps on one input word, with the phase partial(s)
// each step's sign needs (computed from the images before the step)
__device__ __forceinline__ void st_h(Col &A) {
  uint64_t t = A.xd; A.xd = A.zd; A.zd = t;
  t = A.xs; A.xs = A.zs; A.zs = t;
}
__device__ __forceinline__ void st_s(Col &A, int &p) {
  p += pprod(A.zs, A.zd, A.xs, A.xd);  // image(X_a) image(Z_a)
  A.zd ^= A.xd;
  A.zs ^= A.xs;
}
__device__ __forceinline__ void st_cx(Col &A, Col &B, int &p1, int &p2) {
  p1 += pprod(A.zs, A.zd, B.zs, B.zd);  // image(X_c) image(X_t)
  p2 += pprod(A.xs, A.xd, B.xs, B.xd);  // image(Z_c) image(Z_t)
  B.xd ^= A.xd;
  B.xs ^= A.xs;
  A.zd ^= B.zd;
  A.zs ^= B.zs;
}
__device__ __forceinline__ void st_swap(Col &A, Col &B) {
  Col t = A; A = B; B = t;
}

// the gate's bits on one input word (the rest of the 11-gate set by
// composition in circuit order: CZ = H_b CX H_b, CY = S_b^dag CX S_b, ISWAP =
// CZ, SWAP, S_a, S_b); p0..p3 collect the phases in the order gate_signs uses
__device__ __forceinline__ void gate_bits(uint32_t type, Col &A, Col &B, int &p0, int &p1, int &p2,
                                          int &p3) {
  switch (type) {
    case QS_H: st_h(A); break;
    case QS_S: case QS_SDG: st_s(A, p0); break;
    case QS_CX: st_cx(A, B, p0, p1); break;
    case QS_CZ: st_h(B); st_cx(A, B, p0, p1); st_h(B); break;
    case QS_CY: st_s(B, p0); st_cx(A, B, p1, p2); st_s(B, p3); break;
    case QS_SWAP: st_swap(A, B); break;
    case QS_ISWAP: st_h(B); st_cx(A, B, p0, p1); st_h(B); st_swap(A, B); st_s(A, p2); st_s(B, p3); break;
    default: break;  // I, X, Y, Z: signs only
  }
}

// sign steps, replayed by one thread with the reduced phases e[]
struct Signs { int ss[2], sd[2]; bool odd; };

__device__ __forceinline__ void sg_h(Signs &g, int a) {
  int t = g.ss[a]; g.ss[a] = g.sd[a]; g.sd[a] = t;
}
// S^dag X S = -i X Z and S X S^dag = i X Z (Y = i X Z); Z is fixed
__device__ __forceinline__ void sg_s(Signs &g, int a, int e, bool dagger) {
  const int f = (e + (dagger ? 1 : 3)) & 3;
  g.odd |= (f & 1) != 0;
  g.sd[a] ^= g.ss[a] ^ (f >> 1);
}
// CX: X_c -> X_c X_t and Z_t -> Z_c Z_t; both products commute (even phases)
__device__ __forceinline__ void sg_cx(Signs &g, int c, int t, int e1, int e2) {
  g.odd |= ((e1 | e2) & 1) != 0;
  g.sd[c] ^= g.sd[t] ^ (e1 >> 1);
  g.ss[t] ^= g.ss[c] ^ (e2 >> 1);
}
__device__ __forceinline__ void sg_swap(Signs &g) {
  int t = g.ss[0]; g.ss[0] = g.ss[1]; g.ss[1] = t;
  t = g.sd[0]; g.sd[0] = g.sd[1]; g.sd[1] = t;
}

__device__ __forceinline__ void gate_signs(uint32_t type, Signs &g, const int *e) {
  switch (type) {
    case QS_X: g.ss[0] ^= 1; break;                  // X Z X = -Z
    case QS_Z: g.sd[0] ^= 1; break;                  // Z X Z = -X
    case QS_Y: g.ss[0] ^= 1; g.sd[0] ^= 1; break;    // Y anticommutes with X and Z
    case QS_H: sg_h(g, 0); break;
    case QS_S: sg_s(g, 0, e[0], false); break;
    case QS_SDG: sg_s(g, 0, e[0], true); break;
    case QS_CX: sg_cx(g, 0, 1, e[0], e[1]); break;
    case QS_CZ: sg_h(g, 1); sg_cx(g, 0, 1, e[0], e[1]); sg_h(g, 1); break;
    case QS_CY: sg_s(g, 1, e[0], true); sg_cx(g, 0, 1, e[1], e[2]); sg_s(g, 1, e[3], false); break;
    case QS_SWAP: sg_swap(g); break;
    case QS_ISWAP:
      sg_h(g, 1); sg_cx(g, 0, 1, e[0], e[1]); sg_h(g, 1); sg_swap(g);
      sg_s(g, 0, e[2], false); sg_s(g, 1, e[3], false); break;
    default: break;
  }
}

__global__ void __launch_bounds__(256)
inv_gate_layer_kernel(uint64_t *__restrict__ X, uint64_t *__restrict__ Z, uint64_t *__restrict__ qsig,
                      uint32_t n, uint32_t k, uint32_t cs, uint32_t rs,
                      const uint32_t *__restrict__ packed, uint32_t *__restrict__ err) {
  const uint32_t g = blockIdx.x;
  const uint32_t w0 = __ldg(packed + 2 * g), qb = __ldg(packed + 2 * g + 1);
  const uint32_t type = w0 >> 24, qa = w0 & 0xFFFFFFu;
  const bool two = inv_two(type);
  if (qa >= n || type >= QS_NUM_GATE_TYPES || (two && (qb >= n || qb == qa))) {
    if (threadIdx.x == 0) atomicOr(err, kErrBadGate);
    return;
  }
  int p0 = 0, p1 = 0, p2 = 0, p3 = 0;
  if (type >= QS_H) {
    uint64_t *xa = X + (size_t)qa * cs, *za = Z + (size_t)qa * cs;
    uint64_t *xb = X + (size_t)qb * cs, *zb = Z + (size_t)qb * cs;
    for (uint32_t w = threadIdx.x; w < k; w += blockDim.x) {
      Col A = {xa[w], xa[k + w], za[w], za[k + w]};
      Col B = {0, 0, 0, 0};
      if (two) B = {xb[w], xb[k + w], zb[w], zb[k + w]};
      gate_bits(type, A, B, p0, p1, p2, p3);
      xa[w] = A.xd; xa[k + w] = A.xs; za[w] = A.zd; za[k + w] = A.zs;
      if (two) { xb[w] = B.xd; xb[k + w] = B.xs; zb[w] = B.zd; zb[k + w] = B.zs; }
    }
  }
  // block sums of the phase partials (mod 4 suffices)
  __shared__ int sph[4][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int v0 = __reduce_add_sync(0xffffffffu, p0 & 3), v1 = __reduce_add_sync(0xffffffffu, p1 & 3);
  const int v2 = __reduce_add_sync(0xffffffffu, p2 & 3), v3 = __reduce_add_sync(0xffffffffu, p3 & 3);
  if (lane == 0) { sph[0][warp] = v0; sph[1][warp] = v1; sph[2][warp] = v2; sph[3][warp] = v3; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  int e[4];
  for (int j = 0; j < 4; ++j) {
    int v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sph[j][w];
    e[j] = v & 3;
  }
  // signs of the gate's qubits (index 0 = q0, 1 = q1), replayed in step order
  const uint32_t q[2] = {qa, two ? qb : qa};
  Signs sg;
  sg.odd = false;
  for (int i = 0; i < 2; ++i) {
    sg.ss[i] = (int)((qsig[q[i] >> 6] >> (q[i] & 63)) & 1u);
    sg.sd[i] = (int)((qsig[rs + (q[i] >> 6)] >> (q[i] & 63)) & 1u);
  }
  const Signs old = sg;
  gate_signs(type, sg, e);
  if (sg.odd) atomicOr(err, kErrOddPhase);
  const int nq = two ? 2 : 1;
  for (int i = 0; i < nq; ++i) {
    const unsigned long long bit = 1ull << (q[i] & 63);
    if (sg.ss[i] != old.ss[i]) atomicXor(reinterpret_cast<unsigned long long *>(qsig + (q[i] >> 6)), bit);
    if (sg.sd[i] != old.sd[i])
      atomicXor(reinterpret_cast<unsigned long long *>(qsig + rs + (q[i] >> 6)), bit);
  }
}

// qubit signs of a computational basis state: |1> on qubit i is X_i |0>, so
// S_S[i] = initstate[i] and S_D = 0
__global__ void inv_init_signs_kernel(uint64_t *__restrict__ qsig, const uint8_t *__restrict__ init,
                                      uint32_t n, uint32_t rs) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= rs) return;
  uint64_t v = 0;
  if (init != nullptr)
    for (uint32_t b = 0; b < 64; ++b) {
      const uint32_t i = 64 * w + b;
      if (i < n && init[i]) v |= 1ull << b;
    }
  qsig[w] = v;
  qsig[rs + w] = 0;
}

cudaError_t launch_inv_init_signs(const Dev &d, const uint8_t *initstate_dev, cudaStream_t s) {
  inv_init_signs_kernel<<<(d.L.rs + 255) / 256, 256, 0, s>>>(d.qsig, initstate_dev, d.L.n, d.L.rs);
  return cudaGetLastError();
}

cudaError_t launch_inv_gate_layer(const Dev &d, const uint32_t *packed, uint32_t n_gates, cudaStream_t s) {
  if (n_gates == 0) return cudaSuccess;
  const Layout &L = d.L;
  const uint32_t threads = L.k >= 256 ? 256 : (L.k >= 128 ? 128 : (L.k >= 64 ? 64 : 32));
  inv_gate_layer_kernel<<<n_gates, threads, 0, s>>>(d.X, d.Z, d.qsig, L.n, L.k, L.cs, L.rs, packed, d.err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// measurement
// ---------------------------------------------------------------------------
// partials of chunk c: part[(6 c + j) * rs + u], j = 0 Dx, 1 Dz, 2 Fx, 3 Fz, 4 Lx, 5 Lz

// one (row chunk c, word u) of the target pass; pp = pivot (packed row)
__device__ __forceinline__ void inv_targets_item(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ,
                                                 uint32_t rs, uint32_t n, uint32_t k,
                                                 const uint32_t *__restrict__ colx, int64_t pp,
                                                 uint64_t *__restrict__ part, uint32_t rows_per_chunk,
                                                 uint32_t c, uint32_t u) {
  const uint64_t lo = 64ull * k;
  const uint32_t p = (uint32_t)(pp - (int64_t)lo);
  const uint64_t xsp = *(RX + (lo + p) * rs + u), zsp = *(RZ + (lo + p) * rs + u);
  const uint64_t xd0 = *(RX + (uint64_t)p * rs + u), zd0 = *(RZ + (uint64_t)p * rs + u);
  uint64_t dx = 0, dz = 0, fx = 0, fz = 0, lx = 0, lz = 0;
  uint32_t i0 = c * rows_per_chunk;
  const uint32_t i1 = min(n, i0 + rows_per_chunk);
  if (i0 <= p) i0 = p + 1;  // targets come after the pivot
  // the next target at or after row i (stabilizer rows with XS[t][q] = 1)
  auto next = [&](uint32_t i) {
    while (i < i1) {  // a word of column bits at a time
      const uint64_t r = lo + i;
      const uint32_t m = *(colx + (r >> 5)) >> (r & 31);
      if (m) return min(i1, i + (uint32_t)__ffs(m) - 1);
      i += 32 - (uint32_t)(r & 31);
    }
    return i1;
  };
  // the words of the next target are loaded before the current one is
  // stored (distinct rows), so each target costs one memory latency less
  uint32_t t = next(i0);
  uint64_t xs = 0, zs = 0, xd = 0, zd = 0;
  if (t < i1) {
    xs = *(RX + (lo + t) * rs + u); zs = *(RZ + (lo + t) * rs + u);
    xd = *(RX + (uint64_t)t * rs + u); zd = *(RZ + (uint64_t)t * rs + u);
  }
  while (t < i1) {
    const uint32_t t2 = next(t + 1);
    uint64_t nxs = 0, nzs = 0, nxd = 0, nzd = 0;
    if (t2 < i1) {
      nxs = *(RX + (lo + t2) * rs + u); nzs = *(RZ + (lo + t2) * rs + u);
      nxd = *(RX + (uint64_t)t2 * rs + u); nzd = *(RZ + (uint64_t)t2 * rs + u);
    }
    RX[(lo + t) * rs + u] = xs ^ xsp;  // S_t <- S_t S_p (bits)
    RZ[(lo + t) * rs + u] = zs ^ zsp;
    fx ^= xsp & xd & ~(xd0 ^ xs);
    fz ^= zsp & zd & ~(zd0 ^ zs);
    lx ^= xd & dx;  // dx so far: XOR of the chunk's earlier targets
    lz ^= zd & dz;
    dx ^= xd;
    dz ^= zd;
    xs = nxs; zs = nzs; xd = nxd; zd = nzd;
    t = t2;
  }
  uint64_t *o = part + (size_t)6 * c * rs + u;
  o[0] = dx; o[rs] = dz; o[2 * (size_t)rs] = fx; o[3 * (size_t)rs] = fz; o[4 * (size_t)rs] = lx;
  o[5 * (size_t)rs] = lz;
}

// Chunk partials merge in index order: (D, L, F) of an earlier range followed
// by (D', L', F') of a later one is (D ^ D', L ^ L' ^ (D & D'), F ^ F'), the
// pairs across the two ranges being D & D'. A block of 32 warps covers 32
// words (lane = word, coalesced rows of the partials): warp w merges its
// consecutive run of chunks in order, then warp 0 merges the 32 warps' results
// in order. Called by every thread of the block (it holds a block barrier).
constexpr int kCombineWarps = 32;

__device__ __forceinline__ void inv_combine_group(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ,
                                                  uint64_t *__restrict__ qsig, uint32_t rs, uint32_t k,
                                                  int64_t pp, const uint64_t *__restrict__ part,
                                                  uint32_t chunks, uint32_t group,
                                                  uint64_t (*red)[kCombineWarps][32]) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t u = group * 32 + lane;
  const uint32_t per = (chunks + kCombineWarps - 1) / kCombineWarps;
  uint64_t px = 0, pz = 0, fx = 0, fz = 0, lx = 0, lz = 0;
  if (u < rs) {
    const uint32_t c1 = min(chunks, per * (warp + 1));
#pragma unroll 4
    for (uint32_t c = per * warp; c < c1; ++c) {
      const uint64_t *o = part + (size_t)6 * c * rs + u;
      const uint64_t dx = *(o), dz = *(o + rs);
      fx ^= *(o + 2 * (size_t)rs);
      fz ^= *(o + 3 * (size_t)rs);
      lx ^= *(o + 4 * (size_t)rs) ^ (px & dx);
      lz ^= *(o + 5 * (size_t)rs) ^ (pz & dz);
      px ^= dx;
      pz ^= dz;
    }
  }
  red[0][warp][lane] = px; red[1][warp][lane] = pz; red[2][warp][lane] = fx;
  red[3][warp][lane] = fz; red[4][warp][lane] = lx; red[5][warp][lane] = lz;
  __syncthreads();
  if (warp == 0 && u < rs) {
    px = pz = fx = fz = lx = lz = 0;
    for (uint32_t w = 0; w < kCombineWarps; ++w) {
      const uint64_t dx = red[0][w][lane], dz = red[1][w][lane];
      fx ^= red[2][w][lane];
      fz ^= red[3][w][lane];
      lx ^= red[4][w][lane] ^ (px & dx);
      lz ^= red[5][w][lane] ^ (pz & dz);
      px ^= dx;
      pz ^= dz;
    }
    const uint64_t lo = 64ull * k;
    const uint64_t p = (uint64_t)(pp - (int64_t)lo);
    const uint64_t xsp = *(RX + (lo + p) * rs + u), zsp = *(RZ + (lo + p) * rs + u);
    RX[p * rs + u] = *(RX + p * rs + u) ^ px;  // D_p <- D_p prod_t D_t (bits)
    RZ[p * rs + u] = *(RZ + p * rs + u) ^ pz;
    qsig[u] = *(qsig + u) ^ fx ^ (xsp & lx);
    qsig[rs + u] = *(qsig + rs + u) ^ fz ^ (zsp & lz);
  }
}

// One block: the H or H_YZ injection on the pivot, then the X injection when
// S_S[q] differs from the keyed coin; the outcome is the coin. A
// deterministic outcome is S_S[q] (nothing changes). Record, kind, pivot
// reset. Called by every thread of the block.
__device__ __forceinline__ void inv_finalize_block(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ,
                                                   uint64_t *__restrict__ qsig, uint32_t rs, uint32_t k,
                                                   uint32_t q, int64_t pp, int64_t *__restrict__ mst,
                                                   uint64_t midx, uint64_t seed, uint64_t shot,
                                                   uint8_t *__restrict__ record, uint8_t *__restrict__ kinds) {
  const uint32_t tid = threadIdx.x;
  if (pp == kInvNoPivot) {  // deterministic: the outcome is S_S[q]
    if (tid == 0) {
      record[midx] = (uint8_t)((*(qsig + (q >> 6)) >> (q & 63)) & 1u);
      kinds[midx] = 0;
    }
    return;
  }
  const uint64_t lo = 64ull * k;
  const uint64_t p = (uint64_t)(pp - (int64_t)lo);
  uint64_t *xs = RX + (lo + p) * rs, *xd = RX + p * rs, *zs = RZ + (lo + p) * rs, *zd = RZ + p * rs;
  // Y case (the pivot's destabilizer has z at q in the Z_q image): H_YZ, else H
  const bool yz = ((*(xd + (q >> 6)) >> (q & 63)) & 1u) != 0;
  __syncthreads();  // every thread has read xd[q >> 6] before it changes
  for (uint32_t u = tid; u < rs; u += blockDim.x) {
    uint64_t a = *(xs + u), b = *(xd + u), c = *(zs + u), e = *(zd + u);
    uint64_t s0 = *(qsig + u), s1 = *(qsig + rs + u);
    if (yz) {
      s0 ^= a & ~b;
      a ^= b;
      s1 ^= c & ~e;
      c ^= e;
    } else {
      s0 ^= a & b;
      uint64_t t = a; a = b; b = t;
      s1 ^= c & e;
      t = c; c = e; e = t;
    }
    xs[u] = a; xd[u] = b; zs[u] = c; zd[u] = e;
    qsig[u] = s0;
    qsig[rs + u] = s1;
  }
  __syncthreads();
  const uint32_t coin = (uint32_t)(philox4x64_10(midx, shot, 0, 0, seed, kCoinKey).v[0] & 1u);
  const uint32_t sq = (uint32_t)((*(qsig + (q >> 6)) >> (q & 63)) & 1u);
  __syncthreads();  // every thread has read S_S[q] before the X injection changes it
  if (sq != coin)
    for (uint32_t u = tid; u < rs; u += blockDim.x) {
      qsig[u] = *(qsig + u) ^ *(xd + u);
      qsig[rs + u] = *(qsig + rs + u) ^ *(zd + u);
    }
  if (tid == 0) {
    record[midx] = (uint8_t)coin;
    kinds[midx] = 1;
    mst[kMsPivot] = kInvNoPivot;
  }
}

// standalone kernels (one launch per phase; the gather is the CHP path's)
__global__ void __launch_bounds__(256)
inv_targets_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint32_t rs, uint32_t n,
                   uint32_t k, const uint32_t *__restrict__ colx, const int64_t *__restrict__ mst,
                   uint64_t *__restrict__ part, uint32_t rows_per_chunk) {
  const int64_t pp = mst[kMsPivot];
  if (pp == kInvNoPivot) return;
  const uint32_t u = blockIdx.y * blockDim.x + threadIdx.x;
  if (u >= rs) return;
  inv_targets_item(RX, RZ, rs, n, k, colx, pp, part, rows_per_chunk, blockIdx.x, u);
}

__global__ void __launch_bounds__(32 * kCombineWarps)
inv_combine_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint64_t *__restrict__ qsig,
                   uint32_t rs, uint32_t k, const int64_t *__restrict__ mst,
                   const uint64_t *__restrict__ part, uint32_t chunks) {
  __shared__ uint64_t red[6][kCombineWarps][32];  // 48 KB
  const int64_t pp = mst[kMsPivot];
  if (pp == kInvNoPivot) return;
  inv_combine_group(RX, RZ, qsig, rs, k, pp, part, chunks, blockIdx.x, red);
}

__global__ void __launch_bounds__(1024)
inv_finalize_kernel(uint64_t *__restrict__ RX, uint64_t *__restrict__ RZ, uint64_t *__restrict__ qsig,
                    uint32_t rs, uint32_t n, uint32_t k, const uint32_t *__restrict__ qubits, uint32_t qi,
                    int64_t *__restrict__ mst, uint64_t midx, uint64_t seed, uint64_t shot,
                    uint8_t *__restrict__ record, uint8_t *__restrict__ kinds) {
  const uint32_t q = qubits[qi];
  if (q >= n) return;  // flagged by the gather
  inv_finalize_block(RX, RZ, qsig, rs, k, q, mst[kMsPivot], mst, midx, seed, shot, record, kinds);
}

size_t inv_scratch_words(const Layout &L) { return (size_t)6 * kInvChunks * L.rs; }

cudaError_t launch_inv_measure_one(const Dev &d, const uint32_t *qubits, uint32_t i, uint64_t midx,
                                   qs_key key, cudaStream_t s, int *launches) {
  const Layout &L = d.L;
  launch_gather(d, qubits, i, s);
  const uint32_t rows_per_chunk = (L.n + kInvChunks - 1) / kInvChunks;
  const uint32_t chunks = (L.n + rows_per_chunk - 1) / rows_per_chunk;
  const uint32_t tt = std::min<uint32_t>(256, (L.rs + 31) / 32 * 32);  // no idle warps when rs < 256
  inv_targets_kernel<<<dim3(chunks, (L.rs + tt - 1) / tt), tt, 0, s>>>(d.RX, d.RZ, L.rs, L.n, L.k, d.colx,
                                                                      d.mst, d.inv_part, rows_per_chunk);
  inv_combine_kernel<<<(L.rs + 31) / 32, 32 * kCombineWarps, 0, s>>>(d.RX, d.RZ, d.qsig, L.rs, L.k, d.mst,
                                                                    d.inv_part, chunks);
  inv_finalize_kernel<<<1, 1024, 0, s>>>(d.RX, d.RZ, d.qsig, L.rs, L.n, L.k, qubits, i, d.mst, midx,
                                         key.seed, key.shot, d.record, d.kinds);
  if (launches) *launches += 4;
  return cudaGetLastError();
}

}  // namespace qs
