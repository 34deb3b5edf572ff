// FP32-RHS fused interior stage with shared-memory staging (schedule 3).
//
// Same arithmetic as interior_pre_kernel<ORD,true,OCC> (paper Sec. 2 Z4c RHS,
// Sec. 4.3 KO dissipation, Sec. 3 RK stage), organised for GB300:
//
//  Phase A, one field at a time (22 fields, double-buffered): the rows of
//  the field that the tile's stencils touch are brought into shared memory
//  by bulk asynchronous copies (cp.async.bulk through the TMA engine,
//  completion on an mbarrier) while the previous field is being
//  differentiated.  Rows: the tile's z-plane widened by KW in y, the KW
//  planes above and below (tile rows only), and for the eleven fields with
//  mixed second derivatives the pre-pass arrays D_y f (tile rows) and D_z f
//  (tile rows widened by ORD/2 in y); every row is 24 floats starting at
//  storage x = i0 (16-byte aligned).  Each thread evaluates its cell's
//  derivatives, KO dissipation and lopsided advection of the field from
//  shared memory at compile-time offsets and writes them to a per-cell
//  derivative store in shared memory.
//
//  Phase B: the Z4c algebra (rhs_point) reads the derivative store, then the
//  RK stage update and the FP64 enforcement (stage_epilogue) as in the
//  other schedules.
//
// Blocks qualify when their rows are 16-byte aligned and their tiles are
// full: order 6, ghosts 4, n_x % 16 == 0, n_y % 8 == 0, storage x extent and
// block offset multiples of 4 (checked where z4c_create_batch builds the
// tile lists).  Shared memory per CTA: the 158-value derivative store of 128
// cells (81 KB) plus two 9.8 KB stage buffers, so 2 CTAs per SM.
#pragma once

#include "z4c_rhs.cuh"
#include "z4c_tma.cuh"

namespace z4c {

// ---- per-cell derivative store: slot layout ----
// first derivatives are kept for the 16 fields the RHS differentiates once
__host__ __device__ constexpr int d1idx(int f) {
  return f == CHI ? 0 : f == ALPHA ? 1 : f == KHAT ? 2 : f == THETA ? 3
       : (f >= BETAX) ? 4 + (f - BETAX)
       : (f >= GAMX && f <= GAMZ) ? 7 + (f - GAMX)
       : (f >= GXX && f <= GZZ) ? 10 + (f - GXX) : -1;
}
constexpr int SL_VAL = 0;            // 22 centre values (the shadow's minus one added back)
constexpr int SL_D1 = 22;            // 16 fields x 3 directions
constexpr int SL_D2 = 70;            // 11 fields (dslot) x 3 directions
constexpr int SL_MIX = 103;          // 11 fields x (xy, xz, yz)
constexpr int SL_KO = 136;           // 22 KO + advection sums
constexpr int NSLOT = 158;
constexpr int STAGE_NT = TX * TY;    // cells (threads) per tile
constexpr int STAGE_RW = 24;         // floats per staged row

template <int ORD>
struct StageGeom {
  static constexpr int KW = KoAdv<ORD>::KW;      // KO / advection half width
  static constexpr int MW = ORD / 2;             // first-derivative half width
  static constexpr int PK = TY + 2 * KW;         // rows of the tile's own plane
  static constexpr int DYB = PK + 2 * KW * TY;   // first D_y row
  static constexpr int DZB = DYB + TY;           // first D_z row
  static constexpr int NR = DZB + TY + 2 * MW;   // rows with the pre-pass arrays
  static constexpr int NR_PLAIN = DYB;           // rows without them
  static constexpr int BOX = NR * STAGE_RW;      // floats per buffer
  static constexpr size_t SMEM = sizeof(float) * (size_t(NSLOT) * STAGE_NT + 2 * size_t(BOX)) + 2 * sizeof(uint64_t);
};

// Phase-B providers reading the derivative store.
struct StagedSrc {
  const float *ds;
  int tid;
  __device__ __forceinline__ float val(int f) const { return ds[(SL_VAL + f) * STAGE_NT + tid]; }
};
struct StagedDV {
  static constexpr bool kStagedKO = true;
  const float *ds;
  int tid;
  __device__ __forceinline__ float d1(int f, int d) const { return ds[(SL_D1 + 3 * d1idx(f) + d) * STAGE_NT + tid]; }
  __device__ __forceinline__ float d2(int f, int d) const { return ds[(SL_D2 + 3 * dslot(f) + d) * STAGE_NT + tid]; }
  __device__ __forceinline__ float mix(int f, int a, int b) const {
    const int m = (a == 0 && b == 1) ? 0 : (a == 0 && b == 2) ? 1 : 2;
    return ds[(SL_MIX + 3 * dslot(f) + m) * STAGE_NT + tid];
  }
  __device__ __forceinline__ float ko(int f) const { return ds[(SL_KO + f) * STAGE_NT + tid]; }
  // the staged values are already scaled
  __device__ __forceinline__ float d2raw(int f, int d) const { return d2(f, d); }
  __device__ __forceinline__ float mixraw(int f, int a, int b) const { return mix(f, a, b); }
  __device__ __forceinline__ float d2scale() const { return 1.f; }
  __device__ __forceinline__ float mixscale() const { return 1.f; }
};

// centred first / second differences on values p[m-1] = f(+m), q[m-1] = f(-m)
// (the same weights and evaluation order as FD<ORD>::d1 / d2)
template <int ORD>
__device__ __forceinline__ float d1v(const float *p, const float *q) {
  if constexpr (ORD == 6) {
    const float a = p[0] - q[0], b = p[1] - q[1], c = p[2] - q[2];
    return fmaf(a, 45.f, fmaf(b, -9.f, c));
  } else {
    const float a = p[0] - q[0], b = p[1] - q[1];
    return fmaf(a, 8.f, -b);
  }
}
template <int ORD>
__device__ __forceinline__ float d2v(float c0, const float *p, const float *q) {
  if constexpr (ORD == 6) {
    const float a = p[0] + q[0], b = p[1] + q[1], c = p[2] + q[2];
    return fmaf(a, 270.f, fmaf(b, -27.f, fmaf(c, 2.f, c0 * -490.f)));
  } else {
    const float a = p[0] + q[0], b = p[1] + q[1];
    return fmaf(a, 16.f, fmaf(c0, -30.f, -b));
  }
}

// Phase A for field F: derivatives of the staged field at this thread's cell.
// q0 = index of the cell in the tile's plane rows, qz = index of the cell in
// row 0 of the off-plane rows (add the row offset of each plane).
template <int ORD, int F>
__device__ __forceinline__ void stage_field(const float *__restrict__ box, float *__restrict__ ds, int tid,
                                            int q0, int qz, int qdy, int qdz, const bool up[3],
                                            const float ab[3], const Scales<float> &sc) {
  using G = StageGeom<ORD>;
  using K = KoAdv<ORD>;
  constexpr int KW = G::KW, MW = G::MW, RW = STAGE_RW;
  const float c = box[q0];
  // the cross: x[d][m + KW] = f at offset m along d
  float x[3][2 * KW + 1];
#pragma unroll
  for (int m = -KW; m <= KW; ++m) {
    x[0][m + KW] = box[q0 + m];
    x[1][m + KW] = box[q0 + m * RW];
    if (m == 0) {
      x[2][KW] = c;
    } else {
      const int zi = m < 0 ? m + KW : m + KW - 1;  // off-plane index
      x[2][m + KW] = box[qz + zi * TY * RW];
    }
  }
  // centre value (the FP32 shadow stores the shadow_shifted fields minus one)
  ds[(SL_VAL + F) * STAGE_NT + tid] = shadow_shifted(F) ? c + 1.f : c;
  // first derivatives
  constexpr int I1 = d1idx(F);
  constexpr int Q = dslot(F);
  if constexpr (I1 >= 0) {
    float p[MW], q[MW];
#pragma unroll
    for (int m = 1; m <= MW; ++m) {
      p[m - 1] = x[0][KW + m];
      q[m - 1] = x[0][KW - m];
    }
    ds[(SL_D1 + 3 * I1 + 0) * STAGE_NT + tid] = d1v<ORD>(p, q) * sc.s1;
    if constexpr (Q >= 0) {  // y and z from the pre-pass (already times s1)
      ds[(SL_D1 + 3 * I1 + 1) * STAGE_NT + tid] = box[qdy];
      ds[(SL_D1 + 3 * I1 + 2) * STAGE_NT + tid] = box[qdz];
    } else {
#pragma unroll
      for (int d = 1; d < 3; ++d) {
#pragma unroll
        for (int m = 1; m <= MW; ++m) {
          p[m - 1] = x[d][KW + m];
          q[m - 1] = x[d][KW - m];
        }
        ds[(SL_D1 + 3 * I1 + d) * STAGE_NT + tid] = d1v<ORD>(p, q) * sc.s1;
      }
    }
  }
  // second and mixed derivatives
  if constexpr (Q >= 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float p[MW], q[MW];
#pragma unroll
      for (int m = 1; m <= MW; ++m) {
        p[m - 1] = x[d][KW + m];
        q[m - 1] = x[d][KW - m];
      }
      ds[(SL_D2 + 3 * Q + d) * STAGE_NT + tid] = d2v<ORD>(c, p, q) * sc.s2;
    }
    float p[MW], q[MW];
#pragma unroll
    for (int m = 1; m <= MW; ++m) {  // D_x (D_y f)
      p[m - 1] = box[qdy + m];
      q[m - 1] = box[qdy - m];
    }
    ds[(SL_MIX + 3 * Q + 0) * STAGE_NT + tid] = d1v<ORD>(p, q) * sc.s1;
#pragma unroll
    for (int m = 1; m <= MW; ++m) {  // D_x (D_z f)
      p[m - 1] = box[qdz + m];
      q[m - 1] = box[qdz - m];
    }
    ds[(SL_MIX + 3 * Q + 1) * STAGE_NT + tid] = d1v<ORD>(p, q) * sc.s1;
#pragma unroll
    for (int m = 1; m <= MW; ++m) {  // D_y (D_z f)
      p[m - 1] = box[qdz + m * RW];
      q[m - 1] = box[qdz - m * RW];
    }
    ds[(SL_MIX + 3 * Q + 2) * STAGE_NT + tid] = d1v<ORD>(p, q) * sc.s1;
  }
  // KO dissipation and lopsided advection (KoAdv::ko and KoAdv::lop)
  float pairs[KW];
#pragma unroll
  for (int m = 0; m < KW; ++m) pairs[m] = 0.f;
  float adv = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int m = 1; m <= KW; ++m) pairs[m - 1] += x[d][KW + m] + x[d][KW - m];
    float v[K::LN];
#pragma unroll
    for (int qq = 0; qq < K::LN; ++qq) {
      const int m = qq + K::LOFF;
      v[qq] = up[d] ? x[d][KW + m] : x[d][KW - m];
    }
    adv = fmaf(ab[d], K::lop(v), adv);
  }
  ds[(SL_KO + F) * STAGE_NT + tid] = fmaf(K::ko(c, pairs), sc.sko, adv);
}

// Issue the bulk copies of field f's rows into one buffer.  Thread t < rows
// copies row t; thread 0 announces the byte count on the buffer's barrier.
template <int ORD>
__device__ __forceinline__ void stage_issue(const StageArgs &a, const DevBlock &b, const Tile &t, int f,
                                            float *buf, uint64_t *bar, int tid) {
  using G = StageGeom<ORD>;
  constexpr int KW = G::KW, MW = G::MW;
  const int q = dslot(f);
  const int rows = q >= 0 ? G::NR : G::NR_PLAIN;
  if (tid == 0) mbar_arrive_expect_tx(bar, uint32_t(rows * STAGE_RW * sizeof(float)));
  if (tid >= rows) return;
  const int g = b.g, e0 = b.e[0], e1 = b.e[1];
  const int z0 = t.k0 + g, y0 = t.j0 + g, xs = t.i0 + g - KW;
  const float *src;
  int arr, y, z;
  if (tid < G::PK) {
    arr = f; z = z0; y = y0 - KW + tid;
    src = a.x32;
  } else if (tid < G::DYB) {
    const int u = tid - G::PK, zi = u / TY;
    arr = f; z = z0 + (zi < KW ? zi - KW : zi - KW + 1); y = y0 + u % TY;
    src = a.x32;
  } else if (tid < G::DZB) {
    arr = q; z = z0; y = y0 + (tid - G::DYB);
    src = reinterpret_cast<const float *>(a.dstore);
  } else {
    arr = q + NDS; z = z0; y = y0 - MW + (tid - G::DZB);
    src = reinterpret_cast<const float *>(a.dstore);
  }
  src += b.off + (int64_t)arr * b.S + ((int64_t)z * e1 + y) * e0 + xs;
  bulk_g2s(buf + tid * STAGE_RW, src, STAGE_RW * sizeof(float), bar);
}

template <int ORD, int F>
struct StageLoop {
  __device__ __forceinline__ static bool run(const StageArgs &a, const DevBlock &b, const Tile &t, float *box,
                                             uint64_t *bar, float *ds, int tid, int q0, int qz, int qdy, int qdz,
                                             const bool up[3], const float ab[3], const Scales<float> &sc) {
    using G = StageGeom<ORD>;
    constexpr int bi = F & 1;
    float *buf = box + bi * G::BOX;
    const bool ok = mbar_wait(&bar[bi], (F >> 1) & 1);
    if (ok) stage_field<ORD, F>(buf, ds, tid, q0, qz, qdy, qdz, up, ab, sc);
    fence_proxy_async_smem();
    if (__syncthreads_or(!ok)) {
      // give the copies still in flight a bounded time to land, then stop
      mbar_wait(&bar[bi], (F >> 1) & 1, 1u << 16);
      if (F + 1 < NF) mbar_wait(&bar[bi ^ 1], ((F + 1) >> 1) & 1, 1u << 16);
      return false;
    }
    if constexpr (F + 2 < NF) stage_issue<ORD>(a, b, t, F + 2, buf, &bar[bi], tid);
    if constexpr (F + 1 < NF)
      return StageLoop<ORD, F + 1>::run(a, b, t, box, bar, ds, tid, q0, qz, qdy, qdz, up, ab, sc);
    return true;
  }
};

template <int ORD>
__global__ void __launch_bounds__(TX * TY, 2) staged_kernel(StageArgs a, const Tile *__restrict__ tiles) {
  using G = StageGeom<ORD>;
  float *ds = reinterpret_cast<float *>(dyn_smem());
  float *box = ds + NSLOT * STAGE_NT;
  uint64_t *bar = reinterpret_cast<uint64_t *>(box + 2 * G::BOX);
  const Tile t = tiles[blockIdx.x];
  const DevBlock &b = a.blocks[t.block];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int g = b.g, e0 = b.e[0], e1 = b.e[1];
  const int i = t.i0 + tx, j = t.j0 + ty, kk = t.k0;
  const int32_t cidx = ((kk + g) * e1 + (j + g)) * e0 + (i + g);
  const int64_t off = b.off + cidx;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  stage_issue<ORD>(a, b, t, 0, box, &bar[0], tid);
  stage_issue<ORD>(a, b, t, 1, box + G::BOX, &bar[1], tid);

  // loads that do not go through the stage buffers
  const float ichi = inv_chi_f32(a.x64[off], b.chi_floor);
  const Scales<float> sc = scales_of(b, 0.0f);
  bool up[3];
  float ab[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float beta = a.x32[off + (int64_t)(BETAX + d) * b.S];
    up[d] = beta >= 0.f;
    ab[d] = fabsf(beta) * sc.slop;
  }

  // cell position in the buffers (compile-time offsets are added per access)
  constexpr int KW = G::KW, MW = G::MW;
  const int X = tx + KW;  // storage x - (i0 + g - KW)
  const int q0 = (ty + KW) * STAGE_RW + X;
  const int qz = (G::PK + ty) * STAGE_RW + X;
  const int qdy = (G::DYB + ty) * STAGE_RW + X;
  const int qdz = (G::DZB + ty + MW) * STAGE_RW + X;
  if (!StageLoop<ORD, 0>::run(a, b, t, box, bar, ds, tid, q0, qz, qdy, qdz, up, ab, sc)) {
    if (tid == 0 && a.status) atomicOr(a.status, 1);
    return;
  }

  const Phys<float> p{float(b.kappa1), float(b.kappa2), float(b.eta), b.lapse, b.shift};
  const StagedSrc s{ds, tid};
  const StagedDV dv{ds, tid};
  const int st[3] = {1, e0, e0 * e1};
  float k[NF];
  rhs_point<ORD, float>(s, dv, st, sc, p, ichi, k);
  stage_epilogue<float>(a, t.block, off, b.S, k);
}

}  // namespace z4c
