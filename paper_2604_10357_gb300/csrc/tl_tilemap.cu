// Per-tile aggregation maps of the float32 CSR assembly (Sec. 4.4: the
// sparsity pattern is fixed, so where each element entry lands is known
// before the first assembly).
//
// The 32 elements of a tile share nodes: in the structured T10 meshes about
// 44 % of the 3,200 ordered node-pair blocks of a tile repeat a pair that
// another element of the same tile also adds to.  For each tile the map lists
// its distinct (row node I, column slot block) pairs, sorted by CSR position,
// and for each pair the exchange-buffer blocks that contribute to it.  The
// assembly then sums the contributions of a pair in registers and issues one
// reduction per CSR entry and tile instead of one per element entry; the
// lanes of a warp take consecutive pairs, so their reductions fall on
// neighbouring CSR entries.
//
// Map of tile t (fixed capacity kAggCap per tile):
//   agg_nu[t]                 number of distinct pairs U
//   agg_slot[t][u]            {CSR position of row 3I of pair u, row stride 3 deg(I)}
//   agg_cptr[t][u], u <= U    first contribution of pair u (agg_cptr[t][U] = count)
//   agg_code[t][c]            contribution: bits 0-14 the offset of the element's
//                             upper-triangle block in the exchange buffer, bit 15
//                             set when the pair is the transposed block
// Built on the device, one CTA per tile: keys (I << 8 | slot block) with the
// contribution code as payload, bitonic sort in shared memory, then a block
// scan over the heads of equal keys.
#include <algorithm>

#include "tl_internal.cuh"

namespace tl {

namespace {

constexpr int kMapThreads = 512;
constexpr int kKeys = 4096;                  // >= 32 elements x 100 ordered pairs, power of two
constexpr uint32_t kNoKey = 0xffffffffu;
static_assert(kAggCap <= kKeys, "tile map capacity");

// Offset of the upper-triangle block (a, b), a <= b, of element e in the
// exchange buffer: block rows P and 9 - P of warp group P hold 11 blocks of 9
// floats, (P, P..9) then (9-P, 9-P..9).
__device__ __forceinline__ int xchg_offset(int e, int a, int b) {
  const int P = a <= 4 ? a : 9 - a;
  const int j = a <= 4 ? b - a : b + 1;
  return e * 495 + P * 99 + j * 9;
}

__global__ void __launch_bounds__(kMapThreads)
    build_tile_maps(const int32_t* conn, const int32_t* user_of, const uint8_t* blk, const int32_t* node_ptr,
                    int64_t ntiles, int2* agg_slot, uint16_t* agg_cptr, uint16_t* agg_code, int32_t* agg_nu) {
  __shared__ uint32_t key[kKeys];
  __shared__ uint16_t pay[kKeys];
  __shared__ int wsum[kMapThreads / 32];
  __shared__ int s_nu, s_n;
  const int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_nu = 0;
    s_n = 0;
  }
  for (int i = tid; i < kKeys; i += kMapThreads) {
    uint32_t k = kNoKey;
    uint16_t p = 0;
    if (i < kTile * 100) {
      const int e = i / 100, ab = i % 100, a = ab / 10, b = ab % 10;
      const int64_t ge = t * kTile + e;
      if (user_of[ge] >= 0) {
        const uint32_t I = (uint32_t)conn[ge * 10 + a];
        k = (I << 8) | blk[ge * 100 + ab];
        p = (uint16_t)(a <= b ? xchg_offset(e, a, b) : (xchg_offset(e, b, a) | 0x8000));
      }
    }
    key[i] = k;
    pay[i] = p;
  }
  __syncthreads();
  // bitonic sort by key (payload carried along)
  for (int k = 2; k <= kKeys; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < kKeys; i += kMapThreads) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const uint32_t ki = key[i], kj = key[ixj];
          if ((ki > kj) == up) {
            key[i] = kj;
            key[ixj] = ki;
            const uint16_t pi = pay[i];
            pay[i] = pay[ixj];
            pay[ixj] = pi;
          }
        }
      }
      __syncthreads();
    }
  }
  // heads of runs of equal keys -> pair index u (block-wide exclusive scan;
  // thread tid owns entries 8 tid .. 8 tid + 7)
  constexpr int kPer = kKeys / kMapThreads;
  int cnt = 0;
  for (int r = 0; r < kPer; ++r) {
    const int i = tid * kPer + r;
    cnt += key[i] != kNoKey && (i == 0 || key[i] != key[i - 1]);
  }
  int incl = cnt;
  const int lane = tid & 31, w = tid >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int before = 0;
  for (int k = 0; k < w; ++k) before += wsum[k];
  int u = before + incl - cnt;
  int2* slot = agg_slot + t * kAggCap;
  uint16_t* cptr = agg_cptr + t * (kAggCap + 1);
  uint16_t* code = agg_code + t * kAggCap;
  for (int r = 0; r < kPer; ++r) {
    const int i = tid * kPer + r;
    const uint32_t k = key[i];
    if (k == kNoKey) break;                    // sorted: the rest are empty too
    code[i] = pay[i];
    if (i == 0 || k != key[i - 1]) {
      const int I = (int)(k >> 8), b = (int)(k & 0xffu);
      const int p0 = node_ptr[I], p1 = node_ptr[I + 1];
      slot[u] = make_int2(9 * p0 + 3 * b, 3 * (p1 - p0));
      cptr[u] = (uint16_t)i;
      ++u;
    }
    if (i + 1 == kKeys || key[i + 1] == kNoKey) {   // the last entry: totals
      s_n = i + 1;
      s_nu = u;
    }
  }
  __syncthreads();
  if (tid == 0) {
    agg_nu[t] = s_nu;
    cptr[s_nu] = (uint16_t)s_n;
  }
}

}  // namespace

void tile_maps_free(tl_mesh* m);

// Build the maps once per handle (after the pattern); synchronous.  Meshes
// whose node ids do not fit the 24-bit key keep the per-element scatter.
tl_status tile_maps_ensure(tl_mesh* m) {
  if (m->agg_nu) return TL_OK;
  if (m->etype != TL_ELEM_T10) return TL_OK;     // the T10 float32 assembly's maps; ANCF kernels use none
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tile maps need the pattern");
  if (m->nn >= (int64_t(1) << 24)) return fail(m, TL_ERR_INVALID_ARG, "tile maps: more than 2^24 nodes");
  const int64_t ntiles = std::max<int64_t>(m->ne_pad / kTile, 1);
  if (cudaMalloc(&m->agg_slot, sizeof(int2) * kAggCap * ntiles) != cudaSuccess ||
      cudaMalloc(&m->agg_cptr, sizeof(uint16_t) * (kAggCap + 1) * ntiles) != cudaSuccess ||
      cudaMalloc(&m->agg_code, sizeof(uint16_t) * kAggCap * ntiles) != cudaSuccess ||
      cudaMalloc(&m->agg_nu, sizeof(int32_t) * ntiles) != cudaSuccess) {
    tile_maps_free(m);
    return fail(m, TL_ERR_OOM, "tile maps");
  }
  TL_CUDA(m, cudaMemsetAsync(m->agg_nu, 0, sizeof(int32_t) * ntiles, m->stream));
  if (m->ne_pad >= kTile)
    build_tile_maps<<<(unsigned)ntiles, kMapThreads, 0, m->stream>>>(m->d_conn, m->d_user_of, m->d_blk,
                                                                     m->d_node_ptr, ntiles, m->agg_slot,
                                                                     m->agg_cptr, m->agg_code, m->agg_nu);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  TL_CUDA(m, cudaStreamSynchronize(m->stream));
  return TL_OK;
}

void tile_maps_free(tl_mesh* m) {
  void* ptrs[] = {m->agg_slot, m->agg_cptr, m->agg_code, m->agg_nu};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  m->agg_slot = nullptr;
  m->agg_cptr = nullptr;
  m->agg_code = nullptr;
  m->agg_nu = nullptr;
}

}  // namespace tl
