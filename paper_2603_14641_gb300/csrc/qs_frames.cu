// Pauli-frame many-shot sampling, Sec. 5 (Alg. 9).
//
// Frames are two bit matrices X~, Z~ stored per qubit as fw 64-bit shot words
// (bit s of word j = shot 64 j + s), the layout of Alg. 9 with one word
// holding 64 shots of one qubit. Gate layers reuse the column-major gate
// kernel with signs compiled out (qs_gates.cu).
//   Randomize (Alg. 9 init):  X~ = 0; Z~[q][j] = word (j & 3) of
//                             Philox(ctr = (0, q, j >> 2, 1), key = (seed, 0xF4A3E)).
//   MeasureSample (Alg. 9):   out[m][j] = X~[q][j] XOR (ref[m] ? ~0 : 0),
//                             Z~[q][j] = word (j & 3) of Philox(ctr = (m + 1, q, j >> 2, 1), ...).
// The XOR with the reference record is the reading of Alg. 9 that makes the
// output a sample (the frames carry flips relative to one valid record).
//   Noise (frames carry error events, Sec. 3): target i of noise op e in
//                             shot s draws (u, v) = words (2h, 2h + 1) of
//                             Philox(ctr = (e, i, 32 (s >> 6) + (s & 31), 3),
//                             key = (seed, 0xE5505)), h = (s >> 5) & 1.
#include "qs_internal.cuh"

namespace qs {

// fw is a multiple of 4: one Philox block fills 4 consecutive shot words
__global__ void frame_init_kernel(uint64_t *__restrict__ FZ, uint32_t n, uint32_t fw, uint64_t seed) {
  const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t quads = fw >> 2;
  const uint64_t total = (uint64_t)n * quads;
  if (idx >= total) return;
  const uint32_t q = (uint32_t)(idx / quads), j4 = (uint32_t)(idx % quads);
  P4 r = philox4x64_10(0, q, j4, 1, seed, kFrameKey);
  ulonglong2 *p = reinterpret_cast<ulonglong2 *>(FZ + (uint64_t)q * fw + 4ull * j4);
  p[0] = make_ulonglong2(r.v[0], r.v[1]);
  p[1] = make_ulonglong2(r.v[2], r.v[3]);
}

cudaError_t launch_frame_init(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw, uint64_t seed,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(FX, 0, (size_t)n * fw * sizeof(uint64_t), s);
  if (e != cudaSuccess) return e;
  const uint64_t total = (uint64_t)n * (fw >> 2);
  frame_init_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(FZ, n, fw, seed);
  return cudaGetLastError();
}

// grid.x over shot-word quads, grid.y over the measurements of the window
// (the qubits of one launch are distinct)
__global__ void frame_measure_kernel(const uint64_t *__restrict__ FX, uint64_t *__restrict__ FZ,
                                     uint32_t n, uint32_t fw, const uint32_t *__restrict__ qubits,
                                     uint64_t m0, const uint8_t *__restrict__ ref,
                                     uint64_t *__restrict__ out, uint64_t shots, uint64_t seed,
                                     uint32_t *__restrict__ err) {
  const uint32_t i = blockIdx.y;
  const uint32_t j4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (j4 >= (fw >> 2)) return;
  const uint32_t q = qubits[i];
  if (q >= n) {
    if (j4 == 0) atomicOr(err, kErrBadQubit);
    return;
  }
  const uint64_t m = m0 + i;
  const uint64_t ow = (shots + 63) / 64;  // output words per measurement
  const uint64_t flip = ref[m] ? ~0ull : 0ull;
  const uint64_t *fx = FX + (uint64_t)q * fw + 4ull * j4;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const uint64_t j = 4ull * j4 + t;
    if (j < ow) {
      uint64_t v = fx[t] ^ flip;
      if (j == ow - 1 && (shots & 63)) v &= (1ull << (shots & 63)) - 1;
      out[m * ow + j] = v;
    }
  }
  P4 r = philox4x64_10(m + 1, q, j4, 1, seed, kFrameKey);
  ulonglong2 *pz = reinterpret_cast<ulonglong2 *>(FZ + (uint64_t)q * fw + 4ull * j4);
  pz[0] = make_ulonglong2(r.v[0], r.v[1]);
  pz[1] = make_ulonglong2(r.v[2], r.v[3]);
}

cudaError_t launch_frame_measure(uint64_t *FX, uint64_t *FZ, uint32_t n, uint32_t fw,
                                 const uint32_t *qubits, uint32_t count, uint64_t m0,
                                 const uint8_t *ref, uint64_t *out, uint64_t shots, uint64_t seed,
                                 uint32_t *err, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const uint32_t quads = fw >> 2;
  const uint32_t threads = quads < 128 ? ((quads + 31) / 32) * 32 : 128;
  // grid.y is limited to 65535: split long windows
  for (uint32_t off = 0; off < count; off += 65535) {
    const uint32_t c = count - off < 65535 ? count - off : 65535;
    dim3 grid((quads + threads - 1) / threads, c);
    frame_measure_kernel<<<grid, threads, 0, s>>>(FX, FZ, n, fw, qubits + off, m0 + off, ref, out,
                                                  shots, seed, err);
  }
  return cudaGetLastError();
}

// Pauli noise channels on the frames (X_ERROR, Y_ERROR, Z_ERROR, DEPOLARIZE1,
// DEPOLARIZE2; frames carry error events, Sec. 3). One warp per (target, shot
// word j): lane l draws shots 64 j + l and 64 j + 32 + l from one Philox
// block, words (0, 1) and (2, 3) = (u, v) of each, and the warp assembles the
// 64-shot flip words with ballots. Targets of one op are distinct, so every
// frame word has one writer.
__device__ __forceinline__ int noise_code(int kind, uint64_t v) {
  // Pauli code 1 = X, 2 = Y, 3 = Z of a one-qubit channel that fired
  if (kind == QS_NOISE_DEPOLARIZE1) return 1 + (int)__umul64hi(v, 3);
  return kind == QS_NOISE_X ? 1 : kind == QS_NOISE_Y ? 2 : 3;
}
__device__ __forceinline__ uint64_t ballot64(bool lo, bool hi) {
  return (uint64_t)__ballot_sync(0xffffffffu, lo) | ((uint64_t)__ballot_sync(0xffffffffu, hi) << 32);
}
__device__ __forceinline__ bool has_x(int c) { return c == 1 || c == 2; }
__device__ __forceinline__ bool has_z(int c) { return c == 2 || c == 3; }

__global__ void __launch_bounds__(256)
frame_noise_kernel(uint64_t *__restrict__ FX, uint64_t *__restrict__ FZ, uint32_t fw, uint32_t ow,
                   const uint32_t *__restrict__ targets, uint32_t count, uint32_t i0, int kind,
                   uint64_t thr, bool always, uint64_t e, uint64_t seed) {
  const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (wid >= (uint64_t)count * ow) return;  // uniform over the warp
  const uint32_t i = (uint32_t)(wid / ow), j = (uint32_t)(wid % ow);
  const P4 r = philox4x64_10(e, i0 + i, 32ull * j + lane, 3, seed, kNoiseKey);
  const bool f0 = always || r.v[0] < thr, f1 = always || r.v[2] < thr;
  if (kind == QS_NOISE_DEPOLARIZE2) {
    const int k0 = 1 + (int)__umul64hi(r.v[1], 15), k1 = 1 + (int)__umul64hi(r.v[3], 15);
    const int a0 = f0 ? k0 >> 2 : 0, b0 = f0 ? k0 & 3 : 0, a1 = f1 ? k1 >> 2 : 0, b1 = f1 ? k1 & 3 : 0;
    const uint64_t ax = ballot64(has_x(a0), has_x(a1)), az = ballot64(has_z(a0), has_z(a1));
    const uint64_t bx = ballot64(has_x(b0), has_x(b1)), bz = ballot64(has_z(b0), has_z(b1));
    if (lane == 0) {
      const uint64_t qa = targets[2 * i], qb = targets[2 * i + 1];
      if (ax) FX[qa * fw + j] ^= ax;
      if (az) FZ[qa * fw + j] ^= az;
      if (bx) FX[qb * fw + j] ^= bx;
      if (bz) FZ[qb * fw + j] ^= bz;
    }
  } else {
    const int c0 = f0 ? noise_code(kind, r.v[1]) : 0, c1 = f1 ? noise_code(kind, r.v[3]) : 0;
    const uint64_t mx = ballot64(has_x(c0), has_x(c1)), mz = ballot64(has_z(c0), has_z(c1));
    if (lane == 0) {
      const uint64_t q = targets[i];
      if (mx) FX[q * fw + j] ^= mx;
      if (mz) FZ[q * fw + j] ^= mz;
    }
  }
}

cudaError_t launch_frame_noise(uint64_t *FX, uint64_t *FZ, uint32_t fw, uint32_t ow,
                               const uint32_t *targets, uint32_t count, uint32_t i0, int kind,
                               uint64_t thr, bool always, uint64_t e, uint64_t seed,
                               cudaStream_t s) {
  if (count == 0 || ow == 0 || (!always && thr == 0)) return cudaSuccess;  // never fires
  const uint64_t warps = (uint64_t)count * ow;
  const uint64_t blocks = (warps + 7) / 8;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  frame_noise_kernel<<<(unsigned)blocks, 256, 0, s>>>(FX, FZ, fw, ow, targets, count, i0, kind, thr,
                                                      always, e, seed);
  return cudaGetLastError();
}

}  // namespace qs
