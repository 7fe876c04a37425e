// Memory-system probe behind the decision not to fuse gate layers at 180,000
// qubits across a thread-block cluster (one 64-row word slice of every column
// spread over the distributed shared memory of 16 CTAs). A two-qubit gate on
// such a slice reads and writes 16 bytes of a column that, for random qubit
// pairs, sits in another CTA of the cluster 15 times in 16. This probe times
// exactly that access: every thread repeatedly reads and writes 16 bytes in
// its own CTA's shared memory or in a pseudo-randomly chosen other CTA of the
// cluster, and separately the cost of a cluster-wide barrier. Prints one JSON
// object per configuration. Built by build.py next to libqs; run by
// `bench.py --workload dsmemprobe`.
#include <cooperative_groups.h>

#include <cstdint>
#include <cstdio>

namespace cg = cooperative_groups;

constexpr int kSmem = 200 * 1024;
constexpr int kSlots = kSmem / 16;

template <int CL>
__global__ void __launch_bounds__(1024, 1)
dsmem_rmw_kernel(int iters, int sync_every, int remote_pct, unsigned long long *sink) {
  extern __shared__ uint4 buf[];
  cg::cluster_group cluster = cg::this_cluster();
  for (int i = threadIdx.x; i < kSlots; i += blockDim.x) buf[i] = make_uint4(i, 0, 0, 0);
  cluster.sync();
  const unsigned me = cluster.block_rank();
  uint32_t st = threadIdx.x * 2654435761u + me * 97u + 1u;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
    st = st * 1664525u + 1013904223u;  // LCG: rank choice only
    const bool remote = (st & 127u) < (unsigned)remote_pct * 128u / 100u;
    const unsigned rank = remote ? (me + 1 + (st >> 28) % (CL - 1)) % CL : me;
    uint4 *p = cluster.map_shared_rank(buf + (threadIdx.x + (it & 7) * 1024) % kSlots, rank);
    uint4 v = *p;
    v.x ^= st;
    v.y += 1;
    *p = v;
    acc ^= v.x;
    if (sync_every && (it + 1) % sync_every == 0) cluster.sync();
  }
  cluster.sync();  // no CTA leaves while another may still access its shared memory
  if (acc == 0x12345678u) atomicAdd(sink, 1ull);
}

template <int CL>
static int run(int iters, int sync_every, int remote_pct) {
  auto k = dsmem_rmw_kernel<CL>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = kSmem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(CL);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, (void *)k, &cfg) != cudaSuccess || clusters == 0) {
    cudaGetLastError();
    printf("{\"cluster\": %d, \"error\": \"no cluster of this size fits\"}\n", CL);
    return 0;
  }
  cfg.gridDim = dim3(CL * clusters);
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  unsigned long long *sink = nullptr;
  if (cudaMalloc(&sink, 8) != cudaSuccess) return 1;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k, iters, sync_every, remote_pct, sink);  // warm-up
  cudaEventRecord(a);
  if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k, iters, sync_every, remote_pct, sink);
  cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e != cudaSuccess) {
    printf("{\"cluster\": %d, \"error\": \"%s\"}\n", CL, cudaGetErrorString(e));
    return 1;
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  const double ctas = (double)CL * clusters, bytes = 32.0 * iters * 1024.0 * ctas;
  printf("{\"cluster\": %d, \"clusters\": %d, \"iters\": %d, \"sync_every\": %d, \"remote_pct\": %d, "
         "\"ms\": %.4f, \"tb_per_s\": %.3f, \"bytes_per_clk_per_sm\": %.2f, \"us_per_sync\": %.3f}\n",
         CL, clusters, iters, sync_every, remote_pct, ms, bytes / (ms * 1e-3) / 1e12,
         bytes / ctas / (ms * 1e-3) / (clk_khz * 1e3), sync_every ? ms * 1e3 / (iters / sync_every) : 0.0);
  cudaFree(sink);
  return 0;
}

int main() {
  int rc = 0;
  rc |= run<16>(4096, 0, 0);    // every access in the CTA's own shared memory
  rc |= run<16>(4096, 0, 94);   // 15 in 16 in another CTA of a 16-CTA cluster
  rc |= run<8>(4096, 0, 88);    // 7 in 8 in another CTA of an 8-CTA cluster
  rc |= run<16>(4096, 1, 0);    // a cluster barrier after every access: barrier cost
  return rc;
}
