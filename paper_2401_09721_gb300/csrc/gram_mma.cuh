// Patch moments on the tensor pipe (Section 2.3): sum_i a_i a_i^T over patches
// whose entries are small integers (uint8 colours centred on 128, so
// -128..127, exact in float16).  The patches of a batch are staged in shared
// memory entry-major: row r holds entry r of every patch of the batch, and a
// row of constant 1 (for each valid patch) makes sum a and the patch count
// come out of the same product.  One warp-level mma.sync m16n8k16 (float16
// inputs, float32 accumulation) adds 16 patches to a 16 x 8 block of the
// Gram matrix; the same 16 x 16 ldmatrix tile is the A operand of its row
// block and the B operand of two column blocks (A = P^T and B = P read the
// same entry-major rows).
//
// Exactness: every product is at most 2^14 in magnitude and exact in float32;
// the float32 accumulators are moved to int64 before they can exceed 2^22
// (256 patches per accumulator at 2^14 each), so every partial sum is an
// integer far inside float32's 24-bit significand, whatever order the tensor
// pipe adds in.  The int64 totals are exact.
#pragma once

#include <cuda_fp16.h>

#include "fgbd_internal.cuh"

namespace fgbd {

constexpr int kGramFlushPatches = 256;  // patches per accumulator between moves to int64

// four 8x8 float16 tiles from shared memory (addresses of this lane's row)
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// c += A (16x16, row) * B (16x8, col), float16 inputs, float32 accumulation
__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared address of this lane's row for the ldmatrix.x4 of rows [row0, row0 + 16)
// and patches [col0, col0 + 16) of an entry-major block with `stride` halves a row:
// tiles (rows 0-7, patches 0-7), (rows 8-15, 0-7), (rows 0-7, 8-15), (rows 8-15, 8-15),
// i.e. the A fragment of the row block, and the B fragments of its two column
// blocks as registers (0, 2) and (1, 3).
__device__ __forceinline__ uint32_t gram_tile_addr(uint32_t base, int row0, int col0, int stride, int lane) {
  const int row = row0 + (lane & 7) + ((lane >> 3) & 1) * 8;
  const int col = col0 + (lane >> 4) * 8;
  return base + uint32_t(row * stride + col) * 2u;
}

// Move one 16x8 accumulator block (rows 16 mt.., columns 8 nt..) into the
// int64 sums: entry (r, c) with r <= c < De of the Gram matrix of De entries,
// of which entry De - 1 is the constant 1.  s2[r * D + c] for c < D = De - 1,
// s1[r] for c = D (the patch count, r = c = D, is not taken from here).  The
// accumulator is cleared.
__device__ __forceinline__ void gram_flush(float (&c)[4], int mt, int nt, int De, int lane,
                                           unsigned long long* s2, unsigned long long* s1) {
  const int D = De - 1;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int r = 16 * mt + (lane >> 2) + 8 * (e >> 1);
    const int col = 8 * nt + 2 * (lane & 3) + (e & 1);
    const long long v = __float2ll_rz(c[e]);
    c[e] = 0.f;
    if (v == 0 || r > col || r >= D || col > D) continue;
    if (col < D) atomicAdd(&s2[r * D + col], (unsigned long long)v);
    else atomicAdd(&s1[r], (unsigned long long)v);
  }
}

}  // namespace fgbd
