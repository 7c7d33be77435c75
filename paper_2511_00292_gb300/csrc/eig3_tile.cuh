// eig3_tile.cuh -- block-wide, double-buffered staging of array-of-structs
// rows through shared memory with asynchronous 16-byte copies (cp.async), so
// that global loads are coalesced 16-byte accesses that overlap the
// arithmetic of the previous tile.
//
// A tile is kTile consecutive rows of W elements; its byte offset in global
// memory is a multiple of kTile * W * sizeof(E), itself a multiple of 16, so
// for a 16-byte aligned base every full 16-byte chunk of a tile is aligned.
// The chunks go through cp.async.cg (L2 only, no L1 allocation); the ragged
// remainder and misaligned bases use ordinary element loads.  Completion is
// awaited with cp.async.wait_group, a hardware wait on the thread's own
// copies, followed by a block barrier.  Rows are read from shared memory with a
// stride of W elements, free of bank conflicts per half-warp for W = 9 (any
// type) and W = 3, 6 (binary64).
//
// Usage per block (one barrier per tile):
//   tile_issue(first tile -> buffer 0); cp_async_commit();
//   for each tile t of this block:
//     cp_async_wait_all(); __syncthreads();     // tile t landed, tile t-1 done
//     tile_issue(next tile -> other buffer); cp_async_commit();
//     compute tile t from its buffer
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace eig3 {

constexpr int kTile = 256;  // rows per tile = threads per block

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Start copying count elements g[e0 .. e0+count) into s[0 .. count).
template <typename E>
__device__ __forceinline__ void tile_issue(const E *__restrict__ g, int64_t e0, int count,
                                           E *__restrict__ s) {
  const E *src = g + e0;
  int head = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    const int n16 = (count * (int)sizeof(E)) >> 4;
    const char *s8 = reinterpret_cast<const char *>(src);
    char *d8 = reinterpret_cast<char *>(s);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) cp_async16(d8 + 16 * i, s8 + 16 * i);
    head = (n16 << 4) / (int)sizeof(E);
  }
  for (int i = head + threadIdx.x; i < count; i += blockDim.x) s[i] = __ldg(src + i);
}

// Store count elements s[0 .. count) (shared memory, 16-byte aligned) to
// g[e0 .. e0+count) cooperatively: 16-byte vector stores when the destination
// is 16-byte aligned, element stores for the rest.  Rows that are produced
// one per thread and are longer than a few elements (e.g. 27 projector
// entries) are written coalesced this way instead of with a 108-byte stride
// between the lanes of a warp.
template <typename E>
__device__ __forceinline__ void tile_store(const E *__restrict__ s, int count,
                                           E *__restrict__ g, int64_t e0) {
  E *dst = g + e0;
  int head = 0;
  if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
    const int n16 = (count * (int)sizeof(E)) >> 4;
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = s4[i];
    head = (n16 << 4) / (int)sizeof(E);
  }
  for (int i = head + threadIdx.x; i < count; i += blockDim.x) dst[i] = s[i];
}

// The loop above as one call.  Walks the batch of n rows in tiles of kTile
// rows (grid-stride over tiles): the rows of the next tile -- N elements each
// from A and, when M > 0, M elements each from B -- are copied into shared
// memory (sA, sB: two tiles each) while the current one is computed, and
// fn(r0, rows, tileA, tileB) is called once per tile by every thread of the
// block (r0 the tile's first row, rows its row count, tileA/tileB its rows in
// shared memory).  fn may end with a block barrier of its own (e.g. before a
// tile_store of staged outputs); the barrier at the top of the next iteration
// keeps the buffers apart.
template <int N, int M, typename T, typename U, typename Fn>
__device__ __forceinline__ void for_each_tile(const T *__restrict__ A, const U *__restrict__ B,
                                              int64_t n, T (*sA)[kTile * N],
                                              U (*sB)[kTile * (M > 0 ? M : 1)], Fn fn) {
  const int64_t ntiles = (n + kTile - 1) / kTile;
  auto rows_of = [&](int64_t t) { return (int)min((int64_t)kTile, n - t * kTile); };
  auto issue = [&](int64_t t, int b) {
    tile_issue(A, t * kTile * N, rows_of(t) * N, sA[b]);
    if constexpr (M > 0) tile_issue(B, t * kTile * M, rows_of(t) * M, sB[b]);
  };
  int buf = 0;
  if ((int64_t)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  cp_async_commit();
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();  // tile t has landed; every thread is done with the other buffers
    const int64_t tn = t + gridDim.x;
    if (tn < ntiles) issue(tn, buf ^ 1);
    cp_async_commit();
    if constexpr (M > 0) {
      fn(t * kTile, rows_of(t), sA[buf], sB[buf]);
    } else {
      fn(t * kTile, rows_of(t), sA[buf], (const U *)nullptr);
    }
    buf ^= 1;
  }
}

// for_each_tile for one input array, calling body(row_index, row) for every
// row of the batch (row points into shared memory).
template <int N, typename T, typename Body>
__device__ __forceinline__ void for_each_row(const T *__restrict__ A, int64_t n, T (*sA)[kTile * N],
                                             Body body) {
  for_each_tile<N, 0, T, T>(A, (const T *)nullptr, n, sA, (T(*)[kTile])nullptr,
                            [&](int64_t r0, int rows, const T *tile, const T *) {
                              if ((int)threadIdx.x < rows)
                                body(r0 + threadIdx.x, tile + threadIdx.x * N);
                            });
}

// ---------------------------------------------------------------------------
// Warp-granular staging: each warp walks the batch in tiles of 32 rows
// (grid-stride over the grid's warps) with a double buffer of its own in
// shared memory, waiting only on its own copies (cp.async.wait_group, then
// __syncwarp, which also orders the lanes' shared-memory accesses).  No block
// barrier, so the warps of a block drift apart instead of meeting once per
// tile: for the FP64-bound kernels the phases with little binary64 work (the
// seeds of the square roots and the angle, the stores) of different warps
// then overlap the binary64 work of others.  A warp tile starts at element
// 32 W t of its array, a multiple of 16 bytes for W = 3, 6, 9 and 4- or
// 8-byte elements, so its full 16-byte chunks are aligned whenever the base is.
// ---------------------------------------------------------------------------
constexpr int kWarpTile = 32;

template <typename E>
__device__ __forceinline__ void warp_tile_issue(const E *__restrict__ g, int64_t e0, int count,
                                                E *__restrict__ s, int lane) {
  const E *src = g + e0;
  int head = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    const int n16 = (count * (int)sizeof(E)) >> 4;
    const char *s8 = reinterpret_cast<const char *>(src);
    char *d8 = reinterpret_cast<char *>(s);
    for (int i = lane; i < n16; i += 32) cp_async16(d8 + 16 * i, s8 + 16 * i);
    head = (n16 << 4) / (int)sizeof(E);
  }
  for (int i = head + lane; i < count; i += 32) s[i] = __ldg(src + i);
}

// Calls body(i, rowA, rowB) for every row i of the batch that falls to this
// lane: rowA points at the N elements of row i of A in shared memory and rowB
// (M > 0) at the M elements of row i of B.  wA / wB are this warp's two
// buffers (kWarpTile rows each).  Every lane of the warp must call it.
template <int N, int M, typename T, typename U, typename Body>
__device__ __forceinline__ void for_each_row_warp2(const T *__restrict__ A,
                                                   const U *__restrict__ B, int64_t n,
                                                   T (*wA)[kWarpTile * N],
                                                   U (*wB)[kWarpTile * (M > 0 ? M : 1)],
                                                   Body body) {
  const int lane = threadIdx.x & 31;
  const int64_t ntiles = (n + kWarpTile - 1) / kWarpTile;
  const int64_t first = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t step = (int64_t)gridDim.x * (blockDim.x >> 5);
  auto rows_of = [&](int64_t t) { return (int)min((int64_t)kWarpTile, n - t * kWarpTile); };
  auto issue = [&](int64_t t, int b) {
    warp_tile_issue(A, t * kWarpTile * N, rows_of(t) * N, wA[b], lane);
    if constexpr (M > 0) warp_tile_issue(B, t * kWarpTile * M, rows_of(t) * M, wB[b], lane);
  };
  int buf = 0;
  if (first < ntiles) issue(first, 0);
  cp_async_commit();
  for (int64_t t = first; t < ntiles; t += step) {
    cp_async_wait_all();
    __syncwarp();  // tile t has landed; every lane is done with the other buffer
    const int64_t tn = t + step;
    if (tn < ntiles) issue(tn, buf ^ 1);
    cp_async_commit();
    if (lane < rows_of(t)) {
      if constexpr (M > 0) {
        body(t * kWarpTile + lane, wA[buf] + lane * N, wB[buf] + lane * M);
      } else {
        body(t * kWarpTile + lane, wA[buf] + lane * N, (const U *)nullptr);
      }
    }
    buf ^= 1;
  }
}

// One input array: body(i, row).
template <int N, typename T, typename Body>
__device__ __forceinline__ void for_each_row_warp(const T *__restrict__ A, int64_t n,
                                                  T (*wA)[kWarpTile * N], Body body) {
  for_each_row_warp2<N, 0, T, T>(A, (const T *)nullptr, n, wA, (T(*)[kWarpTile])nullptr,
                                 [&](int64_t i, const T *row, const T *) { body(i, row); });
}

}  // namespace eig3
