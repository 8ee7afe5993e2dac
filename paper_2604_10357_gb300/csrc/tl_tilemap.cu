// Per-tile aggregation maps of the float32 CSR assembly (Sec. 4.4: the
// sparsity pattern is fixed, so where each element entry lands is known
// before the first assembly).
//
// The 32 elements of a tile share nodes: in the structured T10 meshes about
// 44 % of a tile's node-pair blocks repeat a pair that another element of
// the same tile also adds to.  The Hessian is stored in full, so the block of
// rows P, columns Q and the block of rows Q, columns P (its transpose) both
// receive every contribution of the node pair {P, Q}.  For each tile the map
// lists its distinct unordered node pairs {P <= Q}, sorted by the CSR
// position of the (P, Q) block, and for each pair the element blocks that
// contribute to it (upper-triangle blocks of the elements, 55 per element).
// The assembly sums a pair's contributions once, in registers, and issues
// one reduction per entry of the (P, Q) block and one per entry of the
// (Q, P) block per tile, instead of one per element entry; the lanes of a
// warp take consecutive pairs, so their reductions fall on neighbouring CSR
// entries.
//
// Map of tile t (fixed capacity kAggCap = 32 x 55 per tile):
//   agg_nu[t]                 number of distinct unordered pairs U
//   agg_slot[t][u]            {CSR position of row 3P of block (P, Q), row stride 3 deg(P),
//                              CSR position of row 3Q of block (Q, P) (-1 when P = Q), 3 deg(Q)}
//   agg_cptr[t][u], u <= U    first contribution of pair u (agg_cptr[t][U] = count);
//                             rows of kAggCptrStride entries (16-byte aligned)
//   agg_code[t][c]            contribution: bits 0-14 the offset of the element's
//                             upper-triangle block (a <= b) in the exchange buffer,
//                             bit 15 set when conn[a] = Q (the block is (Q, P)^T)
// Built on the device, one CTA per tile: keys (P << 8 | slot block of Q in
// P's row) with the contribution code as payload, bitonic sort in shared
// memory, then a block scan over the heads of equal keys; the (Q, P)
// position by a binary search of P in Q's sorted neighbour list.
#include <algorithm>

#include "tl_internal.cuh"

namespace tl {

namespace {

constexpr int kMapThreads = 512;
constexpr int kKeys = 2048;                  // >= 32 elements x 55 upper blocks, power of two
constexpr uint32_t kNoKey = 0xffffffffu;
static_assert(kAggCap <= kKeys, "tile map capacity");

// Upper-triangle block j (0..54) of a 10-node element: (a, b), a <= b, row by row.
__device__ __forceinline__ void upper_block(int j, int& a, int& b) {
  a = 0;
  while (j >= 10 - a) {
    j -= 10 - a;
    ++a;
  }
  b = a + j;
}

__global__ void __launch_bounds__(kMapThreads)
    build_tile_maps(const int32_t* conn, const int32_t* user_of, const uint8_t* blk, const int32_t* node_ptr,
                    const int32_t* node_col, int64_t ntiles, int4* agg_slot, uint16_t* agg_cptr,
                    uint16_t* agg_code, int32_t* agg_nu) {
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
    if (i < kTile * 55) {
      const int e = i / 55;
      int a, b;
      upper_block(i % 55, a, b);
      const int64_t ge = t * kTile + e;
      if (user_of[ge] >= 0) {
        const uint32_t I = (uint32_t)conn[ge * 10 + a], J = (uint32_t)conn[ge * 10 + b];
        if (I <= J) {
          k = (I << 8) | blk[ge * 100 + a * 10 + b];
          p = (uint16_t)xchg_offset(e, a, b);
        } else {
          k = (J << 8) | blk[ge * 100 + b * 10 + a];
          p = (uint16_t)(xchg_offset(e, a, b) | 0x8000);
        }
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
  // thread tid owns entries kPer tid .. kPer tid + kPer - 1)
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
  int4* slot = agg_slot + t * kAggCap;
  uint16_t* cptr = agg_cptr + t * kAggCptrStride;
  uint16_t* code = agg_code + t * kAggCap;
  for (int r = 0; r < kPer; ++r) {
    const int i = tid * kPer + r;
    const uint32_t k = key[i];
    if (k == kNoKey) break;                    // sorted: the rest are empty too
    code[i] = pay[i];
    if (i == 0 || k != key[i - 1]) {
      const int P = (int)(k >> 8), b = (int)(k & 0xffu);
      const int p0 = node_ptr[P], p1 = node_ptr[P + 1];
      const int Q = node_col[p0 + b];
      int4 sl = make_int4(9 * p0 + 3 * b, 3 * (p1 - p0), -1, 0);
      if (Q != P) {
        int lo = node_ptr[Q], hi = node_ptr[Q + 1] - 1;   // P is in Q's sorted list
        const int q0 = lo, q1 = hi + 1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (node_col[mid] < P) lo = mid + 1;
          else hi = mid;
        }
        sl.z = 9 * q0 + 3 * (lo - q0);
        sl.w = 3 * (q1 - q0);
      }
      slot[u] = sl;
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
  if (cudaMalloc(&m->agg_slot, sizeof(int4) * kAggCap * ntiles) != cudaSuccess ||
      cudaMalloc(&m->agg_cptr, sizeof(uint16_t) * kAggCptrStride * ntiles) != cudaSuccess ||
      cudaMalloc(&m->agg_code, sizeof(uint16_t) * kAggCap * ntiles) != cudaSuccess ||
      cudaMalloc(&m->agg_nu, sizeof(int32_t) * ntiles) != cudaSuccess) {
    tile_maps_free(m);
    return fail(m, TL_ERR_OOM, "tile maps");
  }
  TL_CUDA(m, cudaMemsetAsync(m->agg_nu, 0, sizeof(int32_t) * ntiles, m->stream));
  if (m->ne_pad >= kTile)
    build_tile_maps<<<(unsigned)ntiles, kMapThreads, 0, m->stream>>>(m->d_conn, m->d_user_of, m->d_blk,
                                                                     m->d_node_ptr, m->d_node_col, ntiles,
                                                                     m->agg_slot,
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
