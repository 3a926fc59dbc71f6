// Mesh multiplication with interface elements on the device (Sec. 2.4,
// Eq. mmu, Algorithm 3).  The division, the numbering and the coordinate
// rule are stated in include/pdn_mmu.h.
//
// GPU design: no global sort and no hash table.  Every edge (face) of the
// mesh is owned by the lowest (hex, local edge) [(hex, local face)] that has
// it.  A node -> slot CSR (slot = 8 hex + local corner) is built on the device
// and each row sorted; one thread per (hex, local edge) merges the rows of
// the edge's two nodes and takes the first hex in which they are joined by an
// edge (the local edge follows from the two local corners), one thread per
// (hex, local face) merges the rows of two opposite corners and checks the
// other two.  Owner flags and an exclusive scan give each divided edge its
// rank among the owners in (hex, local edge) order, which is the order of
// first appearance of a serial pass; faces likewise.  Children are then written by one thread per
// parent from a 3x3x3 lattice of node ids (3x3 per face for interfaces).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pdn.h"
#include "pdn_mmu.h"

struct pdn_refined {
  int64_t nn = 0, nh = 0, nc = 0, ns = 0, ne = 0, nf = 0;
  int32_t levels = 0;
  double device_ms = 0.0;
  double *X = nullptr;
  int32_t *hex = nullptr, *coh = nullptr, *surf = nullptr;
  int8_t *ply = nullptr;
  uint8_t *fixed = nullptr;
  std::vector<double> ply_angle;
  std::string err;
};

namespace pdn {
namespace {

thread_local std::string g_mmu_error;

// local edges and faces of a hex8 (bottom face counter-clockwise from +z,
// then the top face), and each corner's position in the reference cube in
// half-cells (0 or 2 per axis)
__constant__ int8_t kEdge[12][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}, {4, 5}, {5, 6},
                                    {6, 7}, {7, 4}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
__constant__ int8_t kFace[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4},
                                   {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
__constant__ int8_t kCorner[8][3] = {{0, 0, 0}, {2, 0, 0}, {2, 2, 0}, {0, 2, 0},
                                     {0, 0, 2}, {2, 0, 2}, {2, 2, 2}, {0, 2, 2}};

__device__ __forceinline__ int64_t gid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }

__device__ __forceinline__ void cswap(int32_t &a, int32_t &b) {
  const int32_t lo = a < b ? a : b, hi = a < b ? b : a;
  a = lo;
  b = hi;
}
__device__ __forceinline__ void sort4(int32_t v[4]) {
  cswap(v[0], v[1]);
  cswap(v[2], v[3]);
  cswap(v[0], v[2]);
  cswap(v[1], v[3]);
  cswap(v[1], v[2]);
}

__device__ __forceinline__ void load_hex(const int32_t *hex, int64_t e, int32_t n[8]) {
  const int4 a = reinterpret_cast<const int4 *>(hex)[2 * e];
  const int4 b = reinterpret_cast<const int4 *>(hex)[2 * e + 1];
  n[0] = a.x, n[1] = a.y, n[2] = a.z, n[3] = a.w, n[4] = b.x, n[5] = b.y, n[6] = b.z, n[7] = b.w;
}

// ---------------------------------------------------------------------------
// node -> hex CSR
__global__ void k_mark_surf(const int32_t *surf, int64_t ns, uint8_t *flag) {
  const int64_t i = gid();
  if (i < ns) flag[surf[i]] = 1;
}
__global__ void k_degree(const int32_t *hex, int64_t n8, int32_t *deg) {
  const int64_t t = gid();
  if (t < n8) atomicAdd(&deg[hex[t]], 1);
}
// the rows hold slots 8 hex + local corner; filled in any order, then sorted
// per node, so that the searches below meet the hexes in ascending order
__global__ void k_fill(const int32_t *hex, int64_t n8, int32_t *cursor, int32_t *col) {
  const int64_t t = gid();
  if (t >= n8) return;
  const int32_t pos = atomicAdd(&cursor[hex[t]], 1);
  col[pos] = (int32_t)t;
}
__global__ void k_sort_rows(const int32_t *row, int64_t nn, int32_t *col) {
  const int64_t j = gid();
  if (j >= nn) return;
  const int32_t r0 = row[j], r1 = row[j + 1];
  for (int32_t i = r0 + 1; i < r1; ++i) {
    const int32_t v = col[i];
    int32_t k = i - 1;
    while (k >= r0 && col[k] > v) {
      col[k + 1] = col[k];
      --k;
    }
    col[k + 1] = v;
  }
}

// local edge joining two corners (-1: not an edge), and the face on which
// two corners are diagonal (-1: not diagonal on any face)
__constant__ int8_t kEdgeOf[8][8] = {{-1, 0, -1, 3, 8, -1, -1, -1},  {0, -1, 1, -1, -1, 9, -1, -1},
                                     {-1, 1, -1, 2, -1, -1, 10, -1}, {3, -1, 2, -1, -1, -1, -1, 11},
                                     {8, -1, -1, -1, -1, 4, -1, 7},  {-1, 9, -1, -1, 4, -1, 5, -1},
                                     {-1, -1, 10, -1, -1, 5, -1, 6}, {-1, -1, -1, 11, 7, -1, 6, -1}};
__constant__ int8_t kFaceDiag[8][8] = {{-1, -1, 0, -1, -1, 2, -1, 5}, {-1, -1, -1, 0, 2, -1, 3, -1},
                                       {0, -1, -1, -1, -1, 3, -1, 4}, {-1, 0, -1, -1, 5, -1, 4, -1},
                                       {-1, 2, -1, 5, -1, -1, 1, -1}, {2, -1, 3, -1, -1, -1, -1, 1},
                                       {-1, 3, -1, 4, 1, -1, -1, -1}, {5, -1, 4, -1, -1, 1, -1, -1}};

// first hex (ascending) in which nodes a and b are joined by an edge: its
// code 12 h + local edge, or -1
__device__ int64_t common_edge(const int32_t *row, const int32_t *col, int32_t a, int32_t b) {
  int32_t i = row[a], i1 = row[a + 1], k = row[b], k1 = row[b + 1];
  while (i < i1 && k < k1) {
    const int32_t si = col[i], sk = col[k];
    const int32_t hi = si >> 3, hk = sk >> 3;
    if (hi < hk) {
      ++i;
    } else if (hk < hi) {
      ++k;
    } else {
      const int ed = kEdgeOf[si & 7][sk & 7];
      if (ed >= 0) return 12 * (int64_t)hi + ed;
      ++i;
      ++k;
    }
  }
  return -1;
}

// first hex (ascending) with a face whose node set is {q0, q1, q2, q3} (q0
// and q2 opposite): its code 6 h + local face, or -1.  The hexes holding q0
// and q2 are met in order; where the two are diagonal on a face, the other
// diagonal decides, otherwise all six faces are compared as node sets.
__device__ int64_t common_face(const int32_t *hex, const int32_t *row, const int32_t *col, const int32_t q[4]) {
  int32_t sq[4] = {q[0], q[1], q[2], q[3]};
  sort4(sq);
  int32_t i = row[q[0]], i1 = row[q[0] + 1], k = row[q[2]], k1 = row[q[2] + 1];
  while (i < i1 && k < k1) {
    const int32_t si = col[i], sk = col[k];
    const int32_t hi = si >> 3, hk = sk >> 3;
    if (hi < hk) {
      ++i;
      continue;
    }
    if (hk < hi) {
      ++k;
      continue;
    }
    const int64_t h = hi;
    const int ff = kFaceDiag[si & 7][sk & 7];
    if (ff >= 0) {
      const int c0 = si & 7;
      const bool first = c0 == kFace[ff][0] || c0 == kFace[ff][2];
      const int32_t o1 = hex[8 * h + kFace[ff][first ? 1 : 0]], o3 = hex[8 * h + kFace[ff][first ? 3 : 2]];
      if ((o1 == q[1] && o3 == q[3]) || (o1 == q[3] && o3 == q[1])) return 6 * h + ff;
    } else {
      int32_t n[8];
      load_hex(hex, h, n);
      for (int f2 = 0; f2 < 6; ++f2) {
        int32_t v[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = n[kFace[f2][a]];
        sort4(v);
        if (v[0] == sq[0] && v[1] == sq[1] && v[2] == sq[2] && v[3] == sq[3]) return 6 * h + f2;
      }
    }
    ++i;
    ++k;
  }
  return -1;
}

// ---------------------------------------------------------------------------
// owners: the lowest (hex, local edge) / (hex, local face) with the same
// node set; flag = this position is the owner
__global__ void k_edge_owner(const int32_t *hex, int64_t nh, const int32_t *row, const int32_t *col,
                             int32_t *own, uint8_t *flag) {
  const int64_t t = gid();
  if (t >= 12 * nh) return;
  const int64_t e = t / 12;
  const int k = (int)(t - 12 * e);
  const int32_t a = hex[8 * e + kEdge[k][0]], b = hex[8 * e + kEdge[k][1]];
  // the first hex holding the edge; hex e itself holds it, so one is found
  const int64_t c = common_edge(row, col, a, b);
  const int64_t best = c >= 0 && c < t ? c : t;
  own[t] = (int32_t)best;
  flag[t] = best == t ? 1 : 0;
}

__global__ void k_face_owner(const int32_t *hex, int64_t nh, const int32_t *row, const int32_t *col,
                             int32_t *own, uint8_t *flag) {
  const int64_t t = gid();
  if (t >= 6 * nh) return;
  const int64_t e = t / 6;
  const int f = (int)(t - 6 * e);
  int32_t q[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) q[a] = hex[8 * e + kFace[f][a]];
  const int64_t c = common_face(hex, row, col, q);
  const int64_t best = c >= 0 && c < t ? c : t;
  own[t] = (int32_t)best;
  flag[t] = best == t ? 1 : 0;
}

// ---------------------------------------------------------------------------
// exclusive scan of n small counts into out[0..n], out[n] = total: tiles of
// kScanTile items (8 per thread), tile sums scanned recursively
constexpr int kScanThreads = 256, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

template <typename In>
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const In *in, int64_t n, int32_t *sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
    if (base + i < n) s += (int32_t)in[base + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ int32_t ws[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

template <typename In>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const In *in, int64_t n, const int32_t *offs,
                                                            int32_t *out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  int32_t v[kScanPer], sum = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = base + q < n ? (int32_t)in[base + q] : 0;
    sum += v[q];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __shared__ int32_t ws[kScanThreads / 32];
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    int32_t x = lane < kScanThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane < kScanThreads / 32) ws[lane] = x;
  }
  __syncthreads();
  int32_t ex = (offs ? offs[blockIdx.x] : 0) + (w > 0 ? ws[w - 1] : 0) + inc - sum;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < n) out[base + q] = ex;
    ex += v[q];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[n] = ex;
}

int64_t tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// int32 words of temporary storage a scan of n items needs
int64_t scan_temp(int64_t n) {
  const int64_t nb = tiles(n);
  if (nb <= 1) return 0;
  return nb + (nb + 1) + scan_temp(nb);
}

template <typename In>
cudaError_t scan(const In *in, int64_t n, int32_t *out, int32_t *temp, cudaStream_t s) {
  const int64_t nb = tiles(n);
  if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int32_t), s);
  if (nb == 1) {
    k_tile_scan<In><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
    return cudaGetLastError();
  }
  int32_t *sums = temp, *offs = temp + nb;
  k_tile_sums<In><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan<int32_t>(sums, nb, offs, temp + nb + (nb + 1), s);
  if (e != cudaSuccess) return e;
  k_tile_scan<In><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, offs, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// new nodes
__global__ void k_edge_nodes(const int32_t *hex, int64_t nh, const uint8_t *eflag, const int32_t *eidx,
                             const double *X, int64_t nn, const uint8_t *fixed, const uint8_t *sflag,
                             double *X1, int64_t n1, uint8_t *fixed1, uint8_t *sflag1) {
  const int64_t t = gid();
  if (t >= 12 * nh || !eflag[t]) return;
  const int64_t e = t / 12;
  const int k = (int)(t - 12 * e);
  const int32_t a = hex[8 * e + kEdge[k][0]], b = hex[8 * e + kEdge[k][1]];
  const int64_t j = nn + eidx[t];
#pragma unroll
  for (int i = 0; i < 3; ++i) X1[i * n1 + j] = 0.5 * (X[i * nn + a] + X[i * nn + b]);
  fixed1[j] = fixed[a] & fixed[b];
  sflag1[j] = sflag[a] & sflag[b];
}

__global__ void k_face_nodes(const int32_t *hex, int64_t nh, const uint8_t *fflag, const int32_t *fidx,
                             const double *X, int64_t nn, int64_t ne, const uint8_t *fixed, const uint8_t *sflag,
                             double *X1, int64_t n1, uint8_t *fixed1, uint8_t *sflag1) {
  const int64_t t = gid();
  if (t >= 6 * nh || !fflag[t]) return;
  const int64_t e = t / 6;
  const int f = (int)(t - 6 * e);
  int32_t v[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) v[a] = hex[8 * e + kFace[f][a]];
  const int64_t j = nn + ne + fidx[t];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = X[i * nn + v[0]];
    s = s + X[i * nn + v[1]];
    s = s + X[i * nn + v[2]];
    s = s + X[i * nn + v[3]];
    X1[i * n1 + j] = 0.25 * s;
  }
  fixed1[j] = fixed[v[0]] & fixed[v[1]] & fixed[v[2]] & fixed[v[3]];
  sflag1[j] = sflag[v[0]] & sflag[v[1]] & sflag[v[2]] & sflag[v[3]];
}

// hex centre node and the 8 children
__global__ void k_hex_children(const int32_t *hex, const int8_t *ply, int64_t nh, const int32_t *eown,
                               const int32_t *eidx, const int32_t *fown, const int32_t *fidx, int64_t nn, int64_t ne,
                               int64_t nf, const double *X, const uint8_t *fixed, const uint8_t *sflag, double *X1,
                               int64_t n1, uint8_t *fixed1, uint8_t *sflag1, int32_t *hex1, int8_t *ply1) {
  const int64_t e = gid();
  if (e >= nh) return;
  int32_t n[8];
  load_hex(hex, e, n);
  int32_t L[27];
#pragma unroll
  for (int a = 0; a < 8; ++a) L[kCorner[a][0] + 3 * kCorner[a][1] + 9 * kCorner[a][2]] = n[a];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int p = kEdge[k][0], q = kEdge[k][1];
    const int l = (kCorner[p][0] + kCorner[q][0]) / 2 + 3 * ((kCorner[p][1] + kCorner[q][1]) / 2) +
                  9 * ((kCorner[p][2] + kCorner[q][2]) / 2);
    L[l] = (int32_t)(nn + eidx[eown[12 * e + k]]);
  }
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    int c0 = 0, c1 = 0, c2 = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      c0 += kCorner[kFace[f][a]][0];
      c1 += kCorner[kFace[f][a]][1];
      c2 += kCorner[kFace[f][a]][2];
    }
    L[c0 / 4 + 3 * (c1 / 4) + 9 * (c2 / 4)] = (int32_t)(nn + ne + fidx[fown[6 * e + f]]);
  }
  const int64_t jc = nn + ne + nf + e;
  L[13] = (int32_t)jc;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = X[i * nn + n[0]];
#pragma unroll
    for (int a = 1; a < 8; ++a) s = s + X[i * nn + n[a]];
    X1[i * n1 + jc] = 0.125 * s;
  }
  uint8_t fb = 7, sb = 1;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    fb &= fixed[n[a]];
    sb &= sflag[n[a]];
  }
  fixed1[jc] = fb;
  sflag1[jc] = sb;
  const int8_t p = ply[e];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ci = c & 1, cj = (c >> 1) & 1, ck = c >> 2;
    int32_t out[8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
      out[a] = L[(ci + kCorner[a][0] / 2) + 3 * (cj + kCorner[a][1] / 2) + 9 * (ck + kCorner[a][2] / 2)];
    int4 *dst = reinterpret_cast<int4 *>(hex1) + 2 * (8 * e + c);
    dst[0] = make_int4(out[0], out[1], out[2], out[3]);
    dst[1] = make_int4(out[4], out[5], out[6], out[7]);
    ply1[8 * e + c] = p;
  }
}

// node id of the divided edge {a, b} or face {q0..q3} (q0, q2 opposite) of
// the mesh, from the first hex that has it; -1 when no hex has it
__device__ int32_t find_edge(const int32_t *row, const int32_t *col, const int32_t *eown, const int32_t *eidx,
                             int64_t nn, int32_t a, int32_t b) {
  const int64_t c = common_edge(row, col, a, b);
  return c < 0 ? -1 : (int32_t)(nn + eidx[eown[c]]);
}
__device__ int32_t find_face(const int32_t *hex, const int32_t *row, const int32_t *col, const int32_t *fown,
                             const int32_t *fidx, int64_t nn, int64_t ne, const int32_t q[4]) {
  const int64_t c = common_face(hex, row, col, q);
  return c < 0 ? -1 : (int32_t)(nn + ne + fidx[fown[c]]);
}

// the 4 children of an interface element: both faces divided as hex faces
__global__ void k_coh_children(const int32_t *coh, int64_t nc, const int32_t *hex, const int32_t *row,
                               const int32_t *col, const int32_t *eown, const int32_t *eidx, const int32_t *fown,
                               const int32_t *fidx, int64_t nn, int64_t ne, int32_t *coh1, int32_t *err) {
  const int64_t c = gid();
  if (c >= nc) return;
  // 3x3 lattice of each face: corners (0,0) (2,0) (2,2) (0,2) in face order
  const int qx[4] = {0, 2, 2, 0}, qy[4] = {0, 0, 2, 2};
  int32_t L[2][9];
  bool ok = true;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    int32_t q[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) q[a] = coh[8 * c + 4 * s + a];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      L[s][qx[a] + 3 * qy[a]] = q[a];
      const int b = (a + 1) & 3;
      const int32_t id = find_edge(row, col, eown, eidx, nn, q[a], q[b]);
      ok = ok && id >= 0;
      L[s][(qx[a] + qx[b]) / 2 + 3 * ((qy[a] + qy[b]) / 2)] = id;
    }
    const int32_t id = find_face(hex, row, col, fown, fidx, nn, ne, q);
    ok = ok && id >= 0;
    L[s][4] = id;
  }
  if (!ok) atomicCAS(err, 0, (int32_t)(c + 1));
#pragma unroll
  for (int ch = 0; ch < 4; ++ch) {
    const int ci = ch & 1, cj = ch >> 1;
    int32_t out[8];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 4; ++a) out[4 * s + a] = L[s][(ci + qx[a] / 2) + 3 * (cj + qy[a] / 2)];
    int4 *dst = reinterpret_cast<int4 *>(coh1) + 2 * (4 * c + ch);
    dst[0] = make_int4(out[0], out[1], out[2], out[3]);
    dst[1] = make_int4(out[4], out[5], out[6], out[7]);
  }
}

__global__ void k_surf_new(const uint8_t *sflag_new, int64_t m, const int32_t *pos, int64_t nn, int64_t ns,
                           int32_t *surf1) {
  const int64_t i = gid();
  if (i < m && sflag_new[i]) surf1[ns + pos[i]] = (int32_t)(nn + i);
}

unsigned grid_of(int64_t n, int b) { return (unsigned)std::max<int64_t>(1, (n + b - 1) / b); }

// ---------------------------------------------------------------------------
// one level on device arrays; the inputs are released, the outputs replace
// them in r
struct Level {
  double *X;
  int32_t *hex, *coh, *surf;
  int8_t *ply;
  uint8_t *fixed, *sflag;
  int64_t nn, nh, nc, ns;
};

template <typename P>
cudaError_t dalloc(P **p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  return cudaMalloc(reinterpret_cast<void **>(p), sizeof(P) * (size_t)count);
}

int fail(pdn_refined *r, int code, const std::string &m) {
  r->err = m;
  return code;
}

int divide(pdn_refined *r, Level &in, cudaStream_t s) {
  const int64_t nn = in.nn, nh = in.nh, nc = in.nc, ns = in.ns;
  if (12 * nh > INT32_MAX) return fail(r, PDN_E_ARG, "mesh too large for 32-bit edge positions");
  // phase A buffers
  int32_t *row = nullptr, *cursor = nullptr, *col = nullptr, *eown = nullptr, *eidx = nullptr, *fown = nullptr,
          *fidx = nullptr, *temp = nullptr;
  uint8_t *eflag = nullptr, *fflag = nullptr;
  const int64_t ntemp = std::max({scan_temp(nn + 1), scan_temp(12 * nh), scan_temp(6 * nh), int64_t(1)});
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(dalloc(&row, nn + 2));
  chk(dalloc(&cursor, nn + 1));
  chk(dalloc(&col, 8 * nh));
  chk(dalloc(&eown, 12 * nh));
  chk(dalloc(&eidx, 12 * nh + 1));
  chk(dalloc(&fown, 6 * nh));
  chk(dalloc(&fidx, 6 * nh + 1));
  chk(dalloc(&eflag, 12 * nh));
  chk(dalloc(&fflag, 6 * nh));
  chk(dalloc(&temp, ntemp));
  int32_t *deg = cursor;  // degrees, then scanned into row; cursor reused for the fill
  double *X1 = nullptr;
  int32_t *hex1 = nullptr, *coh1 = nullptr, *surf1 = nullptr, *spos = nullptr, *err = nullptr;
  int8_t *ply1 = nullptr;
  uint8_t *fixed1 = nullptr, *sflag1 = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto &x : ev) chk(cudaEventCreate(&x));
  auto release = [&]() {
    void *ps[] = {row, cursor, col, eown, eidx, fown, fidx, eflag, fflag, temp, spos, err};
    for (void *p : ps)
      if (p) cudaFree(p);
    for (auto &x : ev)
      if (x) cudaEventDestroy(x);
  };
  auto release_out = [&]() {
    void *ps[] = {X1, hex1, coh1, surf1, ply1, fixed1, sflag1};
    for (void *p : ps)
      if (p) cudaFree(p);
  };
  if (e != cudaSuccess) {
    release();
    cudaGetLastError();
    return fail(r, PDN_E_OOM, std::string("mesh multiplication buffers: ") + cudaGetErrorString(e));
  }
  const int B = 256;
  chk(cudaEventRecord(ev[0], s));
  chk(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (nn + 1), s));
  k_degree<<<grid_of(8 * nh, B), B, 0, s>>>(in.hex, 8 * nh, deg);
  chk(cudaGetLastError());
  chk(scan<int32_t>(deg, nn, row, temp, s));
  chk(cudaMemcpyAsync(cursor, row, sizeof(int32_t) * nn, cudaMemcpyDeviceToDevice, s));
  k_fill<<<grid_of(8 * nh, B), B, 0, s>>>(in.hex, 8 * nh, cursor, col);
  chk(cudaGetLastError());
  k_sort_rows<<<grid_of(nn, B), B, 0, s>>>(row, nn, col);
  chk(cudaGetLastError());
  k_edge_owner<<<grid_of(12 * nh, B), B, 0, s>>>(in.hex, nh, row, col, eown, eflag);
  chk(cudaGetLastError());
  k_face_owner<<<grid_of(6 * nh, B), B, 0, s>>>(in.hex, nh, row, col, fown, fflag);
  chk(cudaGetLastError());
  chk(scan<uint8_t>(eflag, 12 * nh, eidx, temp, s));
  chk(scan<uint8_t>(fflag, 6 * nh, fidx, temp, s));
  chk(cudaEventRecord(ev[1], s));
  int32_t tot[2] = {0, 0};
  chk(cudaMemcpyAsync(&tot[0], eidx + 12 * nh, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  chk(cudaMemcpyAsync(&tot[1], fidx + 6 * nh, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) {
    release();
    return fail(r, PDN_E_CUDA, std::string("mesh multiplication (owners): ") + cudaGetErrorString(e));
  }
  const int64_t ne = tot[0], nf = tot[1];
  const int64_t n1 = nn + ne + nf + nh;
  if (n1 > INT32_MAX || 8 * nh > INT32_MAX || 4 * nc > INT32_MAX || ns + (n1 - nn) > INT32_MAX) {
    release();
    return fail(r, PDN_E_ARG, "divided mesh too large for 32-bit node and element ids");
  }
  // phase B buffers
  chk(dalloc(&X1, 3 * n1));
  chk(dalloc(&fixed1, n1));
  chk(dalloc(&sflag1, n1));
  chk(dalloc(&hex1, 64 * nh));
  chk(dalloc(&ply1, 8 * nh));
  chk(dalloc(&coh1, 32 * nc));
  chk(dalloc(&surf1, ns + (n1 - nn)));
  chk(dalloc(&spos, n1 - nn + 1));
  chk(dalloc(&err, 1));
  const int64_t ntemp_b = scan_temp(n1 - nn);
  if (e == cudaSuccess && ntemp_b > ntemp) {
    cudaFree(temp);
    temp = nullptr;
    chk(dalloc(&temp, ntemp_b));
  }
  if (e != cudaSuccess) {
    release();
    release_out();
    cudaGetLastError();
    return fail(r, PDN_E_OOM, std::string("divided mesh: ") + cudaGetErrorString(e));
  }
  chk(cudaEventRecord(ev[2], s));
  chk(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
  for (int i = 0; i < 3; ++i)
    chk(cudaMemcpyAsync(X1 + i * n1, in.X + i * nn, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  chk(cudaMemcpyAsync(fixed1, in.fixed, nn, cudaMemcpyDeviceToDevice, s));
  chk(cudaMemcpyAsync(sflag1, in.sflag, nn, cudaMemcpyDeviceToDevice, s));
  k_edge_nodes<<<grid_of(12 * nh, B), B, 0, s>>>(in.hex, nh, eflag, eidx, in.X, nn, in.fixed, in.sflag, X1, n1,
                                                  fixed1, sflag1);
  chk(cudaGetLastError());
  k_face_nodes<<<grid_of(6 * nh, B), B, 0, s>>>(in.hex, nh, fflag, fidx, in.X, nn, ne, in.fixed, in.sflag, X1, n1,
                                                 fixed1, sflag1);
  chk(cudaGetLastError());
  k_hex_children<<<grid_of(nh, 128), 128, 0, s>>>(in.hex, in.ply, nh, eown, eidx, fown, fidx, nn, ne, nf, in.X,
                                                   in.fixed, in.sflag, X1, n1, fixed1, sflag1, hex1, ply1);
  chk(cudaGetLastError());
  if (nc > 0) {
    k_coh_children<<<grid_of(nc, 128), 128, 0, s>>>(in.coh, nc, in.hex, row, col, eown, eidx, fown, fidx, nn, ne,
                                                     coh1, err);
    chk(cudaGetLastError());
  }
  if (ns > 0) chk(cudaMemcpyAsync(surf1, in.surf, sizeof(int32_t) * ns, cudaMemcpyDeviceToDevice, s));
  chk(scan<uint8_t>(sflag1 + nn, n1 - nn, spos, temp, s));
  k_surf_new<<<grid_of(n1 - nn, B), B, 0, s>>>(sflag1 + nn, n1 - nn, spos, nn, ns, surf1);
  chk(cudaGetLastError());
  chk(cudaEventRecord(ev[3], s));
  int32_t nsn = 0, bad = 0;
  chk(cudaMemcpyAsync(&nsn, spos + (n1 - nn), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  chk(cudaMemcpyAsync(&bad, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  float msa = 0.f, msb = 0.f;
  if (e == cudaSuccess) {
    chk(cudaEventElapsedTime(&msa, ev[0], ev[1]));
    chk(cudaEventElapsedTime(&msb, ev[2], ev[3]));
  }
  release();
  if (e != cudaSuccess) {
    release_out();
    return fail(r, PDN_E_CUDA, std::string("mesh multiplication (division): ") + cudaGetErrorString(e));
  }
  if (bad) {
    release_out();
    return fail(r, PDN_E_ARG, "interface element " + std::to_string(bad - 1) +
                                  ": a face or face edge is not a face or edge of any hex");
  }
  r->device_ms += (double)msa + (double)msb;
  r->ne = ne;
  r->nf = nf;
  void *olds[] = {in.X, in.hex, in.coh, in.surf, in.ply, in.fixed, in.sflag};
  for (void *p : olds)
    if (p) cudaFree(p);
  in.X = X1;
  in.hex = hex1;
  in.coh = coh1;
  in.surf = surf1;
  in.ply = ply1;
  in.fixed = fixed1;
  in.sflag = sflag1;
  in.nn = n1;
  in.nh = 8 * nh;
  in.nc = 4 * nc;
  in.ns = ns + nsn;
  return PDN_OK;
}

}  // namespace
}  // namespace pdn

using namespace pdn;

static int pdn_mesh_multiply_body(pdn_refined **out, const pdn_mesh_desc *m, int32_t ndivi, void *stream) {
  if (!out) return PDN_E_ARG;
  *out = nullptr;
  auto bad = [](int code, const std::string &msg) {
    g_mmu_error = msg;
    return code;
  };
  if (!m || !m->X || !m->hex || m->n_nodes <= 0 || m->n_hex <= 0 || m->n_coh < 0 || m->n_surf < 0)
    return bad(PDN_E_ARG, "mesh: X and hex are required, sizes must be positive");
  if (m->n_coh > 0 && !m->coh) return bad(PDN_E_ARG, "mesh: coh is NULL with n_coh > 0");
  if (m->n_surf > 0 && !m->surf) return bad(PDN_E_ARG, "mesh: surf is NULL with n_surf > 0");
  if (!m->ply_of_hex || !m->ply_angle_deg || m->n_plies < 1 || m->n_plies > 64)
    return bad(PDN_E_ARG, "mesh: ply_of_hex and 1..64 ply angles are required");
  if (ndivi < 0 || ndivi > 6) return bad(PDN_E_ARG, "ndivi must be in 0..6");
  if (m->n_nodes > INT32_MAX || m->n_hex > INT32_MAX / 12 || m->n_coh > INT32_MAX / 8)
    return bad(PDN_E_ARG, "mesh too large for 32-bit ids");
  const int64_t nn = m->n_nodes, nh = m->n_hex, nc = m->n_coh, ns = m->n_surf;
  for (int64_t i = 0; i < 8 * nh; ++i)
    if (m->hex[i] < 0 || m->hex[i] >= nn) return bad(PDN_E_ARG, "hex node id out of range");
  for (int64_t i = 0; i < 8 * nc; ++i)
    if (m->coh[i] < 0 || m->coh[i] >= nn) return bad(PDN_E_ARG, "interface node id out of range");
  for (int64_t i = 0; i < ns; ++i)
    if (m->surf[i] < 0 || m->surf[i] >= nn) return bad(PDN_E_ARG, "surface node id out of range");
  for (int64_t i = 0; i < nh; ++i)
    if (m->ply_of_hex[i] < 0 || m->ply_of_hex[i] >= m->n_plies) return bad(PDN_E_ARG, "ply index out of range");

  pdn_refined *r = new pdn_refined();
  r->levels = ndivi;
  r->ply_angle.assign(m->ply_angle_deg, m->ply_angle_deg + m->n_plies);
  cudaStream_t s = (cudaStream_t)stream;
  Level L{};
  L.nn = nn;
  L.nh = nh;
  L.nc = nc;
  L.ns = ns;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(dalloc(&L.X, 3 * nn));
  chk(dalloc(&L.hex, 8 * nh));
  chk(dalloc(&L.coh, 8 * nc));
  chk(dalloc(&L.surf, ns));
  chk(dalloc(&L.ply, nh));
  chk(dalloc(&L.fixed, nn));
  chk(dalloc(&L.sflag, nn));
  auto free_level = [&]() {
    void *ps[] = {L.X, L.hex, L.coh, L.surf, L.ply, L.fixed, L.sflag};
    for (void *p : ps)
      if (p) cudaFree(p);
  };
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_level();
    delete r;
    return bad(PDN_E_OOM, std::string("mesh upload buffers: ") + cudaGetErrorString(e));
  }
  chk(cudaMemcpyAsync(L.X, m->X, sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(L.hex, m->hex, sizeof(int32_t) * 8 * nh, cudaMemcpyHostToDevice, s));
  if (nc) chk(cudaMemcpyAsync(L.coh, m->coh, sizeof(int32_t) * 8 * nc, cudaMemcpyHostToDevice, s));
  if (ns) chk(cudaMemcpyAsync(L.surf, m->surf, sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(L.ply, m->ply_of_hex, nh, cudaMemcpyHostToDevice, s));
  if (m->fixed)
    chk(cudaMemcpyAsync(L.fixed, m->fixed, nn, cudaMemcpyHostToDevice, s));
  else
    chk(cudaMemsetAsync(L.fixed, 0, nn, s));
  chk(cudaMemsetAsync(L.sflag, 0, nn, s));
  if (ns) {
    k_mark_surf<<<grid_of(ns, 256), 256, 0, s>>>(L.surf, ns, L.sflag);
    chk(cudaGetLastError());
  }
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) {
    free_level();
    delete r;
    return bad(PDN_E_CUDA, std::string("mesh upload: ") + cudaGetErrorString(e));
  }
  for (int lv = 0; lv < ndivi; ++lv) {
    const int rc = divide(r, L, s);
    if (rc) {
      free_level();
      g_mmu_error = "level " + std::to_string(lv + 1) + ": " + r->err;
      delete r;
      return rc;
    }
  }
  r->X = L.X;
  r->hex = L.hex;
  r->coh = L.coh;
  r->surf = L.surf;
  r->ply = L.ply;
  r->fixed = L.fixed;
  cudaFree(L.sflag);
  r->nn = L.nn;
  r->nh = L.nh;
  r->nc = L.nc;
  r->ns = L.ns;
  *out = r;
  return PDN_OK;
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
extern "C" int pdn_mesh_multiply(pdn_refined **out, const pdn_mesh_desc *m, int32_t ndivi, void *stream) {
  try {
    return pdn_mesh_multiply_body(out, m, ndivi, stream);
  } catch (const std::bad_alloc &) {
    g_mmu_error = "host allocation failed";
    return PDN_E_OOM;
  } catch (...) {
    g_mmu_error = "unexpected host error";
    return PDN_E_ARG;
  }
}

extern "C" int pdn_refined_get_info(const pdn_refined *r, pdn_refined_info *info) {
  if (!r || !info) return PDN_E_ARG;
  std::memset(info, 0, sizeof(*info));
  info->n_nodes = r->nn;
  info->n_hex = r->nh;
  info->n_coh = r->nc;
  info->n_surf = r->ns;
  info->n_edges = r->ne;
  info->n_faces = r->nf;
  info->levels = r->levels;
  info->device_ms = r->device_ms;
  return PDN_OK;
}

extern "C" int pdn_refined_get(const pdn_refined *r, double *X, int32_t *hex, int32_t *coh, int8_t *ply_of_hex,
                               uint8_t *fixed, int32_t *surf) {
  if (!r) return PDN_E_ARG;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (X) chk(cudaMemcpy(X, r->X, sizeof(double) * 3 * r->nn, cudaMemcpyDeviceToHost));
  if (hex) chk(cudaMemcpy(hex, r->hex, sizeof(int32_t) * 8 * r->nh, cudaMemcpyDeviceToHost));
  if (coh && r->nc) chk(cudaMemcpy(coh, r->coh, sizeof(int32_t) * 8 * r->nc, cudaMemcpyDeviceToHost));
  if (ply_of_hex) chk(cudaMemcpy(ply_of_hex, r->ply, r->nh, cudaMemcpyDeviceToHost));
  if (fixed) chk(cudaMemcpy(fixed, r->fixed, r->nn, cudaMemcpyDeviceToHost));
  if (surf && r->ns) chk(cudaMemcpy(surf, r->surf, sizeof(int32_t) * r->ns, cudaMemcpyDeviceToHost));
  if (e != cudaSuccess) {
    const_cast<pdn_refined *>(r)->err = std::string("read back: ") + cudaGetErrorString(e);
    return PDN_E_CUDA;
  }
  return PDN_OK;
}

static int pdn_init_refined_body(pdn_ctx **out, const pdn_refined *r, const pdn_material *mat,
                                const pdn_options *opt) {
  if (!out || !r) return PDN_E_ARG;
  *out = nullptr;
  std::vector<double> X(3 * r->nn);
  std::vector<int32_t> hex(8 * r->nh), coh(8 * std::max<int64_t>(r->nc, 1)), surf(std::max<int64_t>(r->ns, 1));
  std::vector<int8_t> ply(r->nh);
  std::vector<uint8_t> fixed(r->nn);
  const int rc = pdn_refined_get(r, X.data(), hex.data(), coh.data(), ply.data(), fixed.data(), surf.data());
  if (rc) return rc;
  pdn_mesh_desc d{};
  d.n_nodes = r->nn;
  d.n_hex = r->nh;
  d.n_coh = r->nc;
  d.n_surf = r->ns;
  d.X = X.data();
  d.hex = hex.data();
  d.coh = r->nc ? coh.data() : nullptr;
  d.ply_of_hex = ply.data();
  d.ply_angle_deg = r->ply_angle.data();
  d.n_plies = (int32_t)r->ply_angle.size();
  d.fixed = fixed.data();
  d.surf = r->ns ? surf.data() : nullptr;
  return pdn_init_mesh(out, &d, mat, opt);
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
extern "C" int pdn_init_refined(pdn_ctx **out, const pdn_refined *r, const pdn_material *mat,
                                const pdn_options *opt) {
  try {
    return pdn_init_refined_body(out, r, mat, opt);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

extern "C" void pdn_refined_destroy(pdn_refined *r) {
  if (!r) return;
  void *ps[] = {r->X, r->hex, r->coh, r->surf, r->ply, r->fixed};
  for (void *p : ps)
    if (p) cudaFree(p);
  delete r;
}

extern "C" const char *pdn_refined_last_error(const pdn_refined *r) {
  return r ? r->err.c_str() : g_mmu_error.c_str();
}
