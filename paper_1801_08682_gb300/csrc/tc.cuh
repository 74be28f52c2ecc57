// tc.cuh -- tensor-core (mma.sync m16n8k8, TF32 in, FP32 accumulate)
// evaluation of the flux divergence of the space-time predictor (Eq. 3):
//   for every space-time node, variable and axis j:
//     G_j[k][c](x) = (1/dx_j) sum_b Dm[x_j][b] F_j[k][c](x with x_j = b)
// Batched across the cells of a tile: along axis j the flux block of a tile
// is a matrix with one row per line (cell, time node k, variable c, the other
// spatial indices) and n columns (b).  One warp multiplies 16 such rows by
// B[b][o] = Dm[o][b] / dx_j (n <= 8, K and N padded to 8 with zeros) and
// writes the 16 x n result back over the rows it read: a row belongs to one
// 16-row block only, so the update is in place and needs no extra storage.
// The node owners store every flux minus the flux of a state that is constant
// over the cell: Dm maps constants to zero, so the derivative is unchanged,
// while TF32 (10-bit mantissa) then rounds only the variation over the cell;
// without the shift a flux of size 1 varying by 0.1 would lose a factor 10 of
// relative accuracy in its derivative.
#pragma once
#include <cstdint>
#include <type_traits>

#include "common.cuh"

namespace aderdg {

__device__ __forceinline__ unsigned smem_u32_tc(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32_16x8x8(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Position of spatial node `node` (x0 + n x1 + n^2 x2) in the flux block of
// axis j when the packed layout is used (n divides 8): axis j runs fastest,
// so lines along j are n consecutive values and a row of 8 values holds 8/n
// whole lines.  Axis 0 keeps the natural order.
template <int n, int d>
__device__ __forceinline__ int tc_pos(int node, int j) {
  if (j == 0) return node;
  const int x0 = node % n, x1 = (node / n) % n, x2 = d == 3 ? node / (n * n) : 0;
  return j == 1 ? x1 + n * x0 + n * n * x2 : x2 + n * x0 + n * n * x1;
}

template <int n>
struct TcPacked {
  static constexpr bool value = n == 2 || n == 4 || n == 8;
};

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *row_addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32_tc(row_addr)));
}

// Packed form (n divides 8).  The block of axis j of one cell is a matrix of
// n m NS / 8 rows of 8 values (L = 8/n lines each); B is the block diagonal
// of L copies of Dm^T / dx_j, so one m16n8k8 step differentiates 16 L lines
// with no padding.  A comes in with one ldmatrix.x4 (16-byte rows: rows of
// 32 bytes, halves at +16), the TF32 operands are the FP32 bits (the tensor
// core ignores the low 13 bits), and the result is stored over the rows
// read.  Each warp takes a contiguous run of 16-row steps, so the next
// operand address is one pointer increment.
template <class K>
__device__ __forceinline__ void tc_flux_divergence_packed(float *Fst, const Tables<float> &T,
                                                          const float (&inv_dx)[3]) {
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, CPB = K::CPB;
  constexpr int BLK = n * m * NS;                // values of one (cell, axis) block
  constexpr int ROWS = BLK / 8;                  // rows of one block
  constexpr int RBB = (ROWS + 15) / 16;          // 16-row steps per block
  constexpr bool FULL = ROWS % 16 == 0;          // no partial step
  constexpr int ITEMS = CPB * RBB;               // steps of one axis in the tile
  constexpr int NWARPS = K::THREADS / 32;
  constexpr int PER = (ITEMS + NWARPS - 1) / NWARPS;
  static_assert(BLK % 8 == 0, "rows of 8 values");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  // ldmatrix row served by this lane: tile = lane / 8 (0: rows 0-7 cols 0-3,
  // 1: rows 8-15 cols 0-3, 2: rows 0-7 cols 4-7, 3: rows 8-15 cols 4-7)
  const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lcol = (lane >> 4) * 4;
  // this warp's contiguous run of steps
  const int it0 = warp * PER, it1 = it0 + PER < ITEMS ? it0 + PER : ITEMS;
#pragma unroll
  for (int j = 0; j < d; ++j) {
    // B[kk][o] = Dm[o % n][kk % n] / dx_j inside the diagonal blocks (o = g)
    uint32_t bf[2];
    bf[0] = to_tf32(t4 / n == g / n ? inv_dx[j] * T.Dm[(g % n) * n + t4 % n] : 0.f);
    bf[1] = to_tf32((t4 + 4) / n == g / n ? inv_dx[j] * T.Dm[(g % n) * n + (t4 + 4) % n] : 0.f);
    int lc = it0 / RBB, rbb = it0 - lc * RBB;
    float *base = Fst + (size_t)(lc * d + j) * BLK + rbb * 128;
    for (int it = it0; it < it1; ++it) {
      const int r_ld = (FULL || rbb * 16 + lrow < ROWS) ? lrow : 0;  // past the block: re-read, not stored
      uint32_t a[4];
      ldmatrix_x4(a, base + r_ld * 8 + lcol);  // TF32 operands: the FP32 bits
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tf32_16x8x8(acc, a, bf);
      __syncwarp();  // every lane's operands are read before any result is written back
      if (FULL || rbb * 16 + g < ROWS) *reinterpret_cast<float2 *>(base + g * 8 + 2 * t4) = make_float2(acc[0], acc[1]);
      if (FULL || rbb * 16 + g + 8 < ROWS)
        *reinterpret_cast<float2 *>(base + (g + 8) * 8 + 2 * t4) = make_float2(acc[2], acc[3]);
      // next step: the next 16 rows, or the first rows of the next cell's block
      if (++rbb == RBB) {
        rbb = 0;
        ++lc;
        base = Fst + (size_t)(lc * d + j) * BLK;
      } else {
        base += 128;
      }
    }
  }
}

// Fst: [CPB][d][n][m][NS] fluxes F_j at the space-time nodes of the tile's
// cells (node = x0 + n x1 + n^2 x2); overwritten by G_j.  All threads of the
// block call this between two block barriers.
template <class K>
__device__ __forceinline__ void tc_flux_divergence(float *Fst, const Tables<float> &T, const float (&inv_dx)[3]) {
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF, CPB = K::CPB;
  static_assert(n <= 8, "one m16n8k8 step covers lines of at most 8 nodes");
  static_assert(std::is_same<typename K::R, float>::value, "TF32 contractions need FP32 predictor data");
  constexpr int ROWS = CPB * n * m * NF;  // lines along one axis in the tile
  constexpr int RB = (ROWS + 15) / 16;
  constexpr int NWARPS = K::THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int j = 0; j < d; ++j) {
    const int s = j == 0 ? 1 : (j == 1 ? n : n * n);  // node stride along axis j
    uint32_t bf[2];
    bf[0] = to_tf32(g < n && t4 < n ? inv_dx[j] * T.Dm[g * n + t4] : 0.f);
    bf[1] = to_tf32(g < n && t4 + 4 < n ? inv_dx[j] * T.Dm[g * n + t4 + 4] : 0.f);
    for (int rb = warp; rb < RB; rb += NWARPS) {
      int base[2];
      bool ok[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = rb * 16 + g + 8 * h;  // row = ((lc n + k) m + c) NF + p
        ok[h] = r < ROWS;
        const int rr = ok[h] ? r : 0;
        const int p = rr % NF, q = rr / NF;  // q = (lc n + k) m + c
        const int c = q % m, lk = q / m;
        const int k = lk % n, lc = lk / n;
        base[h] = (((lc * d + j) * n + k) * m + c) * NS + (p % s) + (p / s) * (s * n);
      }
      uint32_t af[4];
      af[0] = to_tf32(ok[0] && t4 < n ? Fst[base[0] + t4 * s] : 0.f);
      af[1] = to_tf32(ok[1] && t4 < n ? Fst[base[1] + t4 * s] : 0.f);
      af[2] = to_tf32(ok[0] && t4 + 4 < n ? Fst[base[0] + (t4 + 4) * s] : 0.f);
      af[3] = to_tf32(ok[1] && t4 + 4 < n ? Fst[base[1] + (t4 + 4) * s] : 0.f);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tf32_16x8x8(acc, af, bf);
      __syncwarp();  // every lane's operands are read before any result is written back
      const int o0 = 2 * t4, o1 = 2 * t4 + 1;
      if (ok[0] && o0 < n) Fst[base[0] + o0 * s] = acc[0];
      if (ok[0] && o1 < n) Fst[base[0] + o1 * s] = acc[1];
      if (ok[1] && o0 < n) Fst[base[1] + o0 * s] = acc[2];
      if (ok[1] && o1 < n) Fst[base[1] + o1 * s] = acc[3];
    }
  }
}

}  // namespace aderdg
