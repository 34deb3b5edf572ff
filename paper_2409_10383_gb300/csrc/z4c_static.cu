// Constraint norms of one MeshBlock without any device allocation.
//
// For callers that cannot allocate device memory themselves (for example a
// diagnostic hook running inside a host code that owns the whole device
// memory pool, or a monitor that must not allocate while an evolution is in
// flight), the reduction partials of this variant of the constraint kernel
// live in a fixed, file-scope device array instead of caller scratch.  The
// caller still passes the state (input) and receives the norms (output).
//
// The array is shared by every call in the process: each call overwrites the
// records it uses, and calls that overlap on the GPU (different streams or
// threads without ordering) race on it.
#include "z4c.h"
#include "z4c_rhs.cuh"

namespace z4c {
namespace {

constexpr int NPART_S = 8;
constexpr int RESULT_SLOT = Z4C_STATIC_MAX_TILES * NPART_S;  // 6 result values follow the partials

// one record of NPART_S doubles per tile, then the result
__device__ __align__(256) double g_static_scratch[Z4C_STATIC_MAX_TILES * NPART_S + 8];

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// One CTA per TX x TY tile of one z-plane; the tile follows from blockIdx.
template <int ORD>
__global__ void __launch_bounds__(TX * TY) constraints_static_kernel(const double *__restrict__ u, DevBlock b,
                                                                     double r_mask, double *partials) {
  const int tiles_x = (b.n[0] + TX - 1) / TX, tiles_y = (b.n[1] + TY - 1) / TY;
  const int t = blockIdx.x;
  const int kk = t / (tiles_x * tiles_y);
  const int j = (t / tiles_x) % tiles_y * TY + threadIdx.y;
  const int i = t % tiles_x * TX + threadIdx.x;
  double acc[NPART_S] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (i < b.n[0] && j < b.n[1]) {
    const int g = b.g, e0 = b.e[0], e1 = b.e[1];
    const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
    const int st[3] = {1, e0, e0 * e1};
    const Src<double, false> s{u, cidx, b.S};
    const double ichi = 1.0 / fmax(u[cidx], b.chi_floor);
    double out[4];
    constraints_point<ORD>(s, st, scales_of(b, 0.0), ichi, out);
    const double vol = b.h * b.h * b.h;
    const double H = out[0], M2 = out[1] * out[1] + out[2] * out[2] + out[3] * out[3];
    const double x = b.lo[0] + (i + 0.5) * b.h, y = b.lo[1] + (j + 0.5) * b.h, z = b.lo[2] + (kk + 0.5) * b.h;
    const bool far = sqrt(x * x + y * y + z * z) > r_mask;
    acc[0] = H * H * vol;
    acc[1] = M2 * vol;
    acc[2] = vol;
    acc[3] = fabs(H);
    acc[4] = far ? H * H * vol : 0.0;
    acc[5] = far ? M2 * vol : 0.0;
    acc[6] = far ? vol : 0.0;
    acc[7] = sqrt(M2);
  }
  __shared__ double red[NPART_S][TX * TY / 32];
  const int lid = threadIdx.y * TX + threadIdx.x, lane = lid & 31, warp = lid >> 5;
#pragma unroll
  for (int q = 0; q < NPART_S; ++q) {
    const double v = (q == 3 || q == 7) ? wmax(acc[q]) : wsum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (lid == 0) {
#pragma unroll
    for (int q = 0; q < NPART_S; ++q) {
      double v = red[q][0];
      for (int w = 1; w < TX * TY / 32; ++w) v = (q == 3 || q == 7) ? fmax(v, red[q][w]) : v + red[q][w];
      partials[(int64_t)t * NPART_S + q] = v;  // every record this call reads is written here
    }
  }
}

// single CTA, fixed assignment of records to threads (deterministic)
__global__ void constraints_static_finalize(double *scratch, int n) {
  __shared__ double red[NPART_S][32];
  double acc[NPART_S] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < n; i += blockDim.x)
#pragma unroll
    for (int q = 0; q < NPART_S; ++q) {
      const double v = scratch[(int64_t)i * NPART_S + q];
      acc[q] = (q == 3 || q == 7) ? fmax(acc[q], v) : acc[q] + v;
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NPART_S; ++q) {
    const double v = (q == 3 || q == 7) ? wmax(acc[q]) : wsum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[NPART_S];
#pragma unroll
    for (int q = 0; q < NPART_S; ++q) {
      double v = red[q][0];
      for (int w = 1; w < (int)(blockDim.x / 32); ++w) v = (q == 3 || q == 7) ? fmax(v, red[q][w]) : v + red[q][w];
      tot[q] = v;
    }
    double *res = scratch + RESULT_SLOT;
    res[0] = sqrt(tot[0] / tot[2]);
    res[1] = sqrt(tot[1] / tot[2]);
    res[2] = tot[3];
    res[3] = tot[6] > 0 ? sqrt(tot[4] / tot[6]) : 0.0;
    res[4] = tot[6] > 0 ? sqrt(tot[5] / tot[6]) : 0.0;
    res[5] = tot[7];
  }
}

// Device address of g_static_scratch on the current device, looked up on
// every call with that device current (the host-side name is only a
// stand-in for the symbol; the lookup allocates nothing).  Not cached: a
// context torn down and created again may place the array elsewhere.
cudaError_t static_scratch_address(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double *>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace z4c

using namespace z4c;

extern "C" int z4c_constraints_static(const void *u_device, const int32_t n[3], int ghosts, int fd_order,
                                      const double lo[3], double h, double chi_floor, double r_mask,
                                      double *norms, void *cuda_stream) {
  if (!u_device || !n || !lo || !norms) return Z4C_ERR_BAD_ARG;
  if (fd_order != 2 && fd_order != 4 && fd_order != 6) return Z4C_ERR_UNSUPPORTED;
  if (ghosts < fd_order / 2 + 1 || ghosts > 8) return Z4C_ERR_UNSUPPORTED;
  if (!(h > 0.0) || !(chi_floor > 0.0)) return Z4C_ERR_BAD_ARG;
  for (int d = 0; d < 3; ++d)
    if (n[d] < 1) return Z4C_ERR_BAD_ARG;
  const long long tiles = (long long)((n[0] + TX - 1) / TX) * ((n[1] + TY - 1) / TY) * n[2];
  if (tiles > Z4C_STATIC_MAX_TILES) return Z4C_ERR_UNSUPPORTED;  // beyond the fixed scratch
  DevBlock b{};
  const double den1 = fd_order == 2 ? 2.0 : fd_order == 4 ? 12.0 : 60.0;
  const double den2 = fd_order == 2 ? 1.0 : fd_order == 4 ? 12.0 : 180.0;
  for (int d = 0; d < 3; ++d) {
    b.n[d] = n[d];
    b.e[d] = n[d] + 2 * ghosts;
    b.lo[d] = lo[d];
  }
  const long long S = (long long)b.e[0] * b.e[1] * b.e[2];
  if (S * NF >= (1LL << 31)) return Z4C_ERR_UNSUPPORTED;
  b.g = ghosts;
  b.order = fd_order;
  b.S = (int32_t)S;
  b.h = h;
  b.s1 = 1.0 / (den1 * h);
  b.s2 = 1.0 / (den2 * h * h);
  b.smix = 1.0 / (den1 * den1 * h * h);
  b.chi_floor = chi_floor;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double *scratch = nullptr;
  if (static_scratch_address(&scratch) != cudaSuccess) return Z4C_ERR_CUDA;
  const dim3 block(TX, TY);
  if (fd_order == 2)
    constraints_static_kernel<2><<<(unsigned)tiles, block, 0, st>>>((const double *)u_device, b, r_mask, scratch);
  else if (fd_order == 4)
    constraints_static_kernel<4><<<(unsigned)tiles, block, 0, st>>>((const double *)u_device, b, r_mask, scratch);
  else
    constraints_static_kernel<6><<<(unsigned)tiles, block, 0, st>>>((const double *)u_device, b, r_mask, scratch);
  if (cudaGetLastError() != cudaSuccess) return Z4C_ERR_CUDA;
  constraints_static_finalize<<<1, 1024, 0, st>>>(scratch, (int)tiles);
  if (cudaGetLastError() != cudaSuccess) return Z4C_ERR_CUDA;
  double res[6];
  if (cudaMemcpyAsync(res, scratch + RESULT_SLOT, sizeof res, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return Z4C_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return Z4C_ERR_CUDA;
  for (int q = 0; q < 6; ++q) norms[q] = res[q];
  for (int q = 0; q < 6; ++q)
    if (res[q] != res[q]) return Z4C_ERR_NAN;
  return Z4C_OK;
}
