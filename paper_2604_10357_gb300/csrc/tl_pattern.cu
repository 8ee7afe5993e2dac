// Fixed-sparsity pattern, slot map, consistent mass and clamp rows, built
// once per mesh on the device.
//
// Paper: arxiv 2604.10357 Sec. 4.2 (CSR; coefficient-level adjacency from
// element connectivity; the Newton-matrix pattern lifts each adjacent node
// pair (I, J) to a 3x3 DOF block, built once and reused) and Sec. 4.1
// (m_ij = int rho s_i s_j dV, M_e = [m_ij I3], constant).
//
// The paper sorts 64-bit (i, j) keys globally and lifts to DOF level on the
// host.  Here every node gathers the connectivity of its incident elements,
// sorts and de-duplicates it inside one warp (shared memory bitonic sort), and
// the DOF lift is done on the device; the per-element slot map replaces the
// paper's binary search per scattered entry.
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <climits>

#include "tl_internal.cuh"

namespace tl {
namespace {

constexpr int kCap = 2048;          // max candidate neighbours of one node
constexpr int kWarpsPerBlock = 4;

__global__ void count_incidence(const int32_t* conn, const int32_t* user_of, int64_t ne_pad, int nen, int32_t* cnt) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne_pad * nen) return;
  if (user_of[t / nen] < 0) return;
  atomicAdd(&cnt[conn[t]], 1);
}

__global__ void fill_incidence(const int32_t* conn, const int32_t* user_of, int64_t ne_pad, int nen,
                               const int32_t* ptr, int32_t* cursor, int32_t* list) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne_pad * nen) return;
  const int64_t e = t / nen;
  if (user_of[e] < 0) return;
  const int node = conn[t];
  const int slot = atomicAdd(&cursor[node], 1);
  list[ptr[node] + slot] = (int32_t)e;
}

// Warp-wide bitonic sort of buf[0..n), n a power of two.
__device__ void warp_bitonic_sort(int32_t* buf, int n) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n; i += 32) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = buf[i], b = buf[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            buf[i] = b;
            buf[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
}

// One warp per node: gather conn of incident elements (and the nodes that a
// general constraint row couples to it, ex_ptr / ex_col, nullable), sort,
// de-duplicate.
// WRITE = false: deg[node] = number of distinct neighbours.
// WRITE = true : node_col[node_ptr[node] + k] = k-th neighbour (ascending).
template <bool WRITE>
__global__ void node_neighbours(const int32_t* conn, int nen, const int32_t* inc_ptr, const int32_t* inc_list,
                                int64_t nn, int32_t* deg, const int32_t* node_ptr, int32_t* node_col,
                                uint32_t* flags, const int32_t* ex_ptr, const int32_t* ex_col) {
  __shared__ int32_t sbuf[kWarpsPerBlock][kCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t node = blockIdx.x * (int64_t)kWarpsPerBlock + warp;
  if (node >= nn) return;
  int32_t* buf = sbuf[warp];
  const int i0 = inc_ptr[node], i1 = inc_ptr[node + 1];
  const int ne_cand = (i1 - i0) * nen;
  const int x0 = ex_ptr ? ex_ptr[node] : 0, x1 = ex_ptr ? ex_ptr[node + 1] : 0;
  const int ncand = ne_cand + (x1 - x0);
  if (ncand > kCap) {
    if (lane == 0) atomicOr(flags, kFlagBadIndex);
    if (!WRITE && lane == 0) deg[node] = 0;
    return;
  }
  int n = 32;
  while (n < ncand) n <<= 1;
  for (int t = lane; t < n; t += 32) {
    int32_t val = INT_MAX;
    if (t < ne_cand) val = conn[(int64_t)inc_list[i0 + t / nen] * nen + t % nen];
    else if (t < ncand) val = ex_col[x0 + t - ne_cand];
    buf[t] = val;
  }
  __syncwarp();
  warp_bitonic_sort(buf, n);
  int base = WRITE ? node_ptr[node] : 0;
  int count = 0;
  for (int t0 = 0; t0 < n; t0 += 32) {
    const int t = t0 + lane;
    const int32_t val = buf[t];
    const bool keep = (val != INT_MAX) && (t == 0 || buf[t - 1] != val);
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (WRITE && keep) node_col[base + count + __popc(mask & ((1u << lane) - 1u))] = val;
    count += __popc(mask);
  }
  if (!WRITE && lane == 0) deg[node] = count;
}

// DOF CSR: row 3I+d starts at 9 ptr(I) + 3 deg(I) d and lists 3J+e for the
// sorted neighbours J of I.
__global__ void dof_pattern(const int32_t* node_ptr, const int32_t* node_col, int64_t nn, int32_t* row_ptr,
                            int32_t* col) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t node = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp;
  if (node >= nn) return;
  const int p0 = node_ptr[node], p1 = node_ptr[node + 1], deg = p1 - p0;
  if (lane < 3) row_ptr[3 * node + lane] = 9 * p0 + 3 * deg * lane;
  if (node == nn - 1 && lane == 0) row_ptr[3 * nn] = 9 * p1;
  for (int k = lane; k < deg; k += 32) {
    const int J = node_col[p0 + k];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int e = 0; e < 3; ++e) col[9 * p0 + 3 * deg * d + 3 * k + e] = 3 * J + e;
  }
}

__device__ __forceinline__ int find_in_row(const int32_t* node_col, int p0, int p1, int J) {
  int lo = p0, hi = p1 - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = node_col[mid];
    if (v == J) return mid - p0;
    if (v < J) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// blk[e][a*nen+b] = position of conn[e][b] in the adjacency of conn[e][a].
__global__ void slot_blocks(const int32_t* conn, int64_t ne_pad, int nen, const int32_t* node_ptr,
                            const int32_t* node_col, uint8_t* blk, uint32_t* flags) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nen2 = nen * nen;
  if (t >= ne_pad * nen2) return;
  const int64_t e = t / nen2;
  const int ab = (int)(t % nen2), a = ab / nen, b = ab % nen;
  const int I = conn[e * nen + a], J = conn[e * nen + b];
  const int k = find_in_row(node_col, node_ptr[I], node_ptr[I + 1], J);
  if (k < 0 || k > 255) {
    atomicOr(flags, kFlagBadIndex);
    blk[t] = 0;
    return;
  }
  blk[t] = (uint8_t)k;
}

__constant__ double c_mass420_d[10][10] = {
    {6, 1, 1, 1, -4, -6, -4, -4, -6, -6},     {1, 6, 1, 1, -4, -4, -6, -6, -4, -6},
    {1, 1, 6, 1, -6, -4, -4, -6, -6, -4},     {1, 1, 1, 6, -6, -6, -6, -4, -4, -4},
    {-4, -4, -6, -6, 32, 16, 16, 16, 16, 8},  {-6, -4, -4, -6, 16, 32, 16, 8, 16, 16},
    {-4, -6, -4, -6, 16, 16, 32, 16, 8, 16},  {-4, -6, -6, -4, 16, 8, 16, 32, 16, 16},
    {-6, -4, -6, -4, 16, 16, 8, 16, 32, 16},  {-6, -6, -4, -4, 8, 16, 16, 16, 16, 32}};

// Consistent mass M_IJ of T10 elements (node level, same pattern as the
// adjacency) and its row sums, for the real elements of one material segment.
__global__ void assemble_mass(const int32_t* conn, const double* geo64, const uint8_t* blk, const int32_t* node_ptr,
                              int64_t e_begin, int64_t e_end, double rho, double* mass, double* mrow) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t e = e_begin + t / 100;
  if (e >= e_end) return;
  const int ab = (int)(t % 100), a = ab / 10, b = ab % 10;
  const double m = rho * geo64[e * 16 + 12] * c_mass420_d[a][b] / 420.0;
  const int I = conn[e * 10 + a];
  atomicAdd(&mass[node_ptr[I] + blk[e * 100 + ab]], m);
  atomicAdd(&mrow[I], m);
}

__global__ void fixed_diag(const int32_t* fixed, int64_t nfixed, const int32_t* node_ptr, const int32_t* node_col,
                           int32_t* diag, uint32_t* flags) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nfixed) return;
  const int I = fixed[j];
  const int p0 = node_ptr[I], p1 = node_ptr[I + 1], deg = p1 - p0;
  const int k = find_in_row(node_col, p0, p1, I);
  if (k < 0) atomicOr(flags, kFlagBadIndex);
  for (int d = 0; d < 3; ++d) diag[3 * j + d] = 9 * p0 + 3 * deg * d + 3 * k + d;
}

__global__ void expand_slots(const int32_t* conn, int nen, const uint8_t* blk, const int32_t* node_ptr,
                             const int32_t* user_of, int64_t ne_pad, int32_t* slot_map) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nd = 3 * nen, nd2 = nd * nd;
  if (t >= ne_pad * nd2) return;
  const int64_t e = t / nd2;
  const int ue = user_of[e];
  if (ue < 0) return;
  const int rs = (int)(t % nd2), r = rs / nd, s = rs % nd;
  const int a = r / 3, i = r % 3, b = s / 3, k = s % 3;
  const int I = conn[e * nen + a];
  const int p0 = node_ptr[I], deg = node_ptr[I + 1] - p0;
  slot_map[(int64_t)ue * nd2 + rs] = 9 * p0 + 3 * deg * i + 3 * blk[e * nen * nen + a * nen + b] + k;
}

inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

tl_status build_pattern(tl_mesh* m, const int32_t* fixed_nodes, int64_t nfixed) {
  cudaStream_t s = m->stream;
  const int64_t nn = m->nn, ne_pad = m->ne_pad;
  // ---- fixed nodes (host validation) ------------------------------------
  std::vector<int32_t> fixed(fixed_nodes, fixed_nodes + nfixed);
  std::sort(fixed.begin(), fixed.end());
  for (int64_t j = 0; j < nfixed; ++j) {
    if (fixed[j] < 0 || fixed[j] >= nn) return fail(m, TL_ERR_INVALID_ARG, "fixed node id out of range");
    if (j > 0 && fixed[j] == fixed[j - 1]) return fail(m, TL_ERR_INVALID_ARG, "duplicate fixed node id");
  }
  std::vector<int32_t> fixed_of(nn, -1);
  for (int64_t j = 0; j < nfixed; ++j) fixed_of[fixed[j]] = (int32_t)j;

  int32_t *d_cnt = nullptr, *d_inc_ptr = nullptr, *d_cursor = nullptr, *d_inc = nullptr, *d_deg = nullptr,
          *d_fixed = nullptr, *d_ex_ptr = nullptr, *d_ex_col = nullptr;
  void* d_tmp = nullptr;
  size_t tmp_bytes = 0;
  tl_status st = TL_OK;
  auto cleanup = [&]() {
    cudaFree(d_cnt);
    cudaFree(d_inc_ptr);
    cudaFree(d_cursor);
    cudaFree(d_inc);
    cudaFree(d_deg);
    cudaFree(d_fixed);
    cudaFree(d_tmp);
    cudaFree(d_ex_ptr);
    cudaFree(d_ex_col);
  };
#define TRY(call)                                   \
  do {                                              \
    cudaError_t _e = (call);                        \
    if (_e != cudaSuccess) {                        \
      st = cuda_fail(m, _e, #call);                 \
      cleanup();                                    \
      return st;                                    \
    }                                               \
  } while (0)

  const int nen = m->nen;
  const int64_t ninc = m->ne * nen;
  TRY(cudaMalloc(&d_cnt, sizeof(int32_t) * (nn + 1)));
  TRY(cudaMalloc(&d_inc_ptr, sizeof(int32_t) * (nn + 1)));
  TRY(cudaMalloc(&d_cursor, sizeof(int32_t) * (nn + 1)));
  TRY(cudaMalloc(&d_inc, sizeof(int32_t) * std::max<int64_t>(ninc, 1)));
  TRY(cudaMalloc(&d_deg, sizeof(int32_t) * (nn + 1)));
  TRY(cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * (nn + 1), s));
  TRY(cudaMemsetAsync(d_cursor, 0, sizeof(int32_t) * (nn + 1), s));
  TRY(cudaMemsetAsync(m->d_flags, 0, sizeof(uint32_t), s));
  count_incidence<<<nblocks(ne_pad * nen, 256), 256, 0, s>>>(m->d_conn, m->d_user_of, ne_pad, nen, d_cnt);
  TRY(cudaGetLastError());
  // exclusive scan of (nn + 1) counts (the last count is 0) -> pointers
  TRY(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, d_cnt, d_inc_ptr, (int)(nn + 1), s));
  TRY(cudaMalloc(&d_tmp, tmp_bytes));
  TRY(cub::DeviceScan::ExclusiveSum(d_tmp, tmp_bytes, d_cnt, d_inc_ptr, (int)(nn + 1), s));
  fill_incidence<<<nblocks(ne_pad * nen, 256), 256, 0, s>>>(m->d_conn, m->d_user_of, ne_pad, nen, d_inc_ptr,
                                                            d_cursor, d_inc);
  TRY(cudaGetLastError());
  // ---- neighbours: count, scan, write ------------------------------------
  if (m->ncon > 0) {   // node pairs coupled by general constraint rows (the Sec. 4.2 fill)
    TRY(cudaMalloc(&d_ex_ptr, sizeof(int32_t) * (nn + 1)));
    TRY(cudaMalloc(&d_ex_col, sizeof(int32_t) * std::max<size_t>(m->h_ex_col.size(), 1)));
    TRY(cudaMemcpyAsync(d_ex_ptr, m->h_ex_ptr.data(), sizeof(int32_t) * (nn + 1), cudaMemcpyHostToDevice, s));
    if (!m->h_ex_col.empty())
      TRY(cudaMemcpyAsync(d_ex_col, m->h_ex_col.data(), sizeof(int32_t) * m->h_ex_col.size(),
                          cudaMemcpyHostToDevice, s));
  }
  TRY(cudaMemsetAsync(d_deg, 0, sizeof(int32_t) * (nn + 1), s));
  node_neighbours<false><<<nblocks(nn, kWarpsPerBlock), 32 * kWarpsPerBlock, 0, s>>>(
      m->d_conn, nen, d_inc_ptr, d_inc, nn, d_deg, nullptr, nullptr, m->d_flags, d_ex_ptr, d_ex_col);
  TRY(cudaGetLastError());
  TRY(cudaMalloc(&m->d_node_ptr, sizeof(int32_t) * (nn + 1)));
  size_t tmp2 = 0;
  TRY(cub::DeviceScan::ExclusiveSum(nullptr, tmp2, d_deg, m->d_node_ptr, (int)(nn + 1), s));
  if (tmp2 > tmp_bytes) {
    TRY(cudaFree(d_tmp));
    d_tmp = nullptr;
    TRY(cudaMalloc(&d_tmp, tmp2));
    tmp_bytes = tmp2;
  }
  TRY(cub::DeviceScan::ExclusiveSum(d_tmp, tmp_bytes, d_deg, m->d_node_ptr, (int)(nn + 1), s));
  int32_t nnz_node = 0;
  uint32_t flags = 0;
  TRY(cudaMemcpyAsync(&nnz_node, m->d_node_ptr + nn, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TRY(cudaMemcpyAsync(&flags, m->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  if (flags & kFlagBadIndex) {
    cleanup();
    return fail(m, TL_ERR_UNSUPPORTED, "a node has more than 2,048 neighbour candidates (nen per incident "
                                       "element plus its constraint couplings)");
  }
  const int64_t nnz = 9 * (int64_t)nnz_node;
  if (nnz >= (int64_t)INT_MAX) {
    cleanup();
    return fail(m, TL_ERR_OVERFLOW, "nnz of the Hessian does not fit in int32");
  }
  m->nnz_node = nnz_node;
  m->nnz = nnz;
  TRY(cudaMalloc(&m->d_node_col, sizeof(int32_t) * std::max<int64_t>(nnz_node, 1)));
  node_neighbours<true><<<nblocks(nn, kWarpsPerBlock), 32 * kWarpsPerBlock, 0, s>>>(
      m->d_conn, nen, d_inc_ptr, d_inc, nn, d_deg, m->d_node_ptr, m->d_node_col, m->d_flags, d_ex_ptr, d_ex_col);
  TRY(cudaGetLastError());
  // ---- DOF pattern --------------------------------------------------------
  TRY(cudaMalloc(&m->d_row_ptr, sizeof(int32_t) * (3 * nn + 1)));
  TRY(cudaMalloc(&m->d_col, sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
  dof_pattern<<<nblocks(nn, 8), 256, 0, s>>>(m->d_node_ptr, m->d_node_col, nn, m->d_row_ptr, m->d_col);
  TRY(cudaGetLastError());
  // ---- slot blocks -------------------------------------------------------
  TRY(cudaMalloc(&m->d_blk, (size_t)nen * nen * std::max<int64_t>(ne_pad, 1)));
  slot_blocks<<<nblocks(ne_pad * nen * nen, 256), 256, 0, s>>>(m->d_conn, ne_pad, nen, m->d_node_ptr,
                                                              m->d_node_col, m->d_blk, m->d_flags);
  TRY(cudaGetLastError());
  // ---- mass --------------------------------------------------------------
  TRY(cudaMalloc(&m->d_mass, sizeof(double) * std::max<int64_t>(nnz_node, 1)));
  TRY(cudaMalloc(&m->d_mrow, sizeof(double) * nn));
  TRY(cudaMemsetAsync(m->d_mass, 0, sizeof(double) * std::max<int64_t>(nnz_node, 1), s));
  TRY(cudaMemsetAsync(m->d_mrow, 0, sizeof(double) * nn, s));
  if (m->etype == TL_ELEM_T10) {
    for (const Segment& sg : m->segs) {
      const int64_t cnt = (sg.end - sg.begin) * 100;
      if (cnt == 0) continue;
      assemble_mass<<<nblocks(cnt, 256), 256, 0, s>>>(m->d_conn, m->d_geo64, m->d_blk, m->d_node_ptr, sg.begin,
                                                     sg.end, m->mats[sg.mat].rho, m->d_mass, m->d_mrow);
      TRY(cudaGetLastError());
    }
  } else {
    const tl_status ms = ancf_build_mass(m);    // exact mass, gravity weights, element mass table
    if (ms != TL_OK) {
      cleanup();
      return ms;
    }
  }
  {
    const tl_status ms = mass_split_build(m, s);     // float32 pairs of the mass (double-float residual)
    if (ms != TL_OK) {
      cleanup();
      return ms;
    }
  }
  // ---- clamp rows --------------------------------------------------------
  m->nfixed = nfixed;
  TRY(cudaMalloc(&m->d_fixed_of_node, sizeof(int32_t) * nn));
  TRY(cudaMemcpyAsync(m->d_fixed_of_node, fixed_of.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s));
  TRY(cudaMalloc(&m->d_fixed_diag, sizeof(int32_t) * std::max<int64_t>(3 * nfixed, 1)));
  if (nfixed > 0) {
    TRY(cudaMalloc(&d_fixed, sizeof(int32_t) * nfixed));
    TRY(cudaMemcpyAsync(d_fixed, fixed.data(), sizeof(int32_t) * nfixed, cudaMemcpyHostToDevice, s));
    fixed_diag<<<nblocks(nfixed, 128), 128, 0, s>>>(d_fixed, nfixed, m->d_node_ptr, m->d_node_col, m->d_fixed_diag,
                                                   m->d_flags);
    TRY(cudaGetLastError());
  }
  TRY(cudaMemcpyAsync(&flags, m->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  cleanup();
#undef TRY
  if (flags & kFlagBadIndex) return fail(m, TL_ERR_UNSUPPORTED, "a node has more than 256 neighbours");
  m->have_pattern = true;
  return TL_OK;
}

tl_status expand_slot_map(const tl_mesh* m, int32_t* slot_map, cudaStream_t s) {
  const int nd = 3 * m->nen;
  expand_slots<<<nblocks(m->ne_pad * nd * nd, 256), 256, 0, s>>>(m->d_conn, m->nen, m->d_blk, m->d_node_ptr,
                                                                m->d_user_of, m->ne_pad, slot_map);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}

}  // namespace tl
