// GPU twin of the cell-body generator in synth.c (input generation only; it
// holds none of the rendering method's arithmetic). Same recipe: a jittered
// grid of cells, a sphere per present cell with its interior value inside
// radius r and the membrane value 230 within r + 2, background 20, plus
// Gaussian noise of sigma 8 drawn per voxel by Box-Muller from the same
// counter-based hash, rounded and clamped to u8. Distances and the noise are
// FP32 here (FP64 on the CPU), so a small fraction of voxels -- on a sphere
// boundary, or where the noisy value lands within rounding of .5 -- can
// differ from the CPU generator; the cell parameters are the CPU's own.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// uniform in [0, 1) from the top 24 bits of the hash of (seed, stream, ctr)
__device__ __forceinline__ float u01f(uint64_t seed, uint64_t stream, uint64_t ctr) {
  const uint64_t h = mix64(mix64(seed ^ (stream * 0xd1b54a32d192ed03ULL)) ^ ctr);
  return (float)(uint32_t)(h >> 40) * (1.0f / 16777216.0f);
}

__global__ void k_cells(uint8_t* __restrict__ out, long N, uint64_t seed, long z0, long nz, int cell,
                        const float4* __restrict__ table, long ng) {
  const long total = N * N * nz;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long x = i % N, y = (i / N) % N, z = z0 + i / (N * N);
    const long gx = x / cell, gy = y / cell, gz = z / cell;
    const float px = (float)x + 0.5f, py = (float)y + 0.5f, pz = (float)z + 0.5f;
    float v = 20.0f;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b)
        for (int c = -1; c <= 1; ++c) {
          const long X = gx + c, Y = gy + b, Z = gz + a;
          if (X < 0 || Y < 0 || Z < 0 || X >= ng || Y >= ng || Z >= ng) continue;
          const float4* t = table + 2 * ((Z * ng + Y) * ng + X);
          const float4 p = __ldg(t), q = __ldg(t + 1);
          if (p.x == 0.0f) continue;
          const float dx = px - p.y, dy = py - p.z, dz = pz - p.w;
          const float d = sqrtf(dx * dx + dy * dy + dz * dz);
          const float w = d < q.x ? q.y : (d < q.x + 2.0f ? 230.0f : 0.0f);
          v = fmaxf(v, w);
        }
    const uint64_t idx = ((uint64_t)z * N + y) * N + x;
    const float u1 = fmaxf(u01f(seed, 8, idx), 1.0f / 33554432.0f), u2 = u01f(seed, 9, idx);
    v += 8.0f * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    const float r = floorf(v + 0.5f);
    out[(size_t)(i)] = (uint8_t)fminf(fmaxf(r, 0.0f), 255.0f);
  }
}

}  // namespace

// Fills dev_out (device memory, nz * N * N voxels, x fastest) with slices
// z0 .. z0 + nz - 1 of the cell-body volume of edge N. host_table is
// sy_cell_table's output. Returns a cudaError_t value (0 on success); waits
// for the work to finish.
extern "C" int sy_cells_u8_gpu(uint8_t* dev_out, long N, uint64_t seed, long z0, long nz, int cell,
                               const float* host_table, long ng) {
  float4* table = nullptr;
  const size_t bytes = (size_t)ng * ng * ng * 8 * sizeof(float);
  cudaError_t e = cudaMalloc(&table, bytes);
  if (e != cudaSuccess) return (int)e;
  e = cudaMemcpy(table, host_table, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_cells<<<sms * 16, 256>>>(dev_out, N, seed, z0, nz, cell, table, ng);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  cudaFree(table);
  return (int)e;
}
