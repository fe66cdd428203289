// Droplet topology of the current state on the GPU (TLBfind, arXiv 2109.12565, Sec. 2.4):
// droplet regions (rho_1 above a threshold), their labels and centres of mass, the digital
// Voronoi tessellation coloured by the nearest centre, the Delaunay links read off the points
// where digital Voronoi cells meet, and the T1 (diagonal flip) events between two analyses.
//
// Definitions (the same as the oracle's):
//   D1  droplet node: fluid node with rho_1 > B_th;
//   D2  4-neighbour connectivity, x periodic, y periodic when periodic_y;
//   D3  droplet ids 0, 1, ... in the order of each droplet's smallest node index y * nx + x;
//   D4  centre = plain mean of the node coordinates, unwrapped relative to the smallest node;
//   D5  Voronoi colour = id of the nearest centre (double, unfused dx*dx + dy*dy, minimum image,
//       ties to the smaller id), -1 at solid nodes;
//   D6  links: 2 x 2 windows with three colours give the three pairs, with four colours the four
//       pairs of neighbouring corners.
//
// Pipeline (all on the caller's stream, no host round trip until the counts are read; the
// per-droplet kernels take the droplet count from the workspace header the labelling wrote; the
// launch sequence is captured once per workspace, bound, threshold and buffer into a CUDA graph):
//   rho_1 (MODE_RHO1: the field mode's rho_1, from the 9 planes of component 1) -> reset of the
//   accumulators -> labels: union-find with atomicMin hooks, so every root ends as its component's
//   smallest node, first inside 32 x 32 tiles in shared memory, then across the tile borders -> ids:
//   root bits per 32 nodes and a scan of their counts -> centres: 64-bit integer sums of the
//   unwrapped offsets (exact, order independent) -> cell grid of the centres -> colours: nearest
//   staged centre, screened in FP32 and settled in FP64 near Voronoi edges -> links: a bounded
//   adjacency set per droplet (atomicCAS), sorted per droplet in a warp, compacted by a scan.
//   Every result is independent of thread scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "lb_host.h"

namespace tlb {
namespace drops {

constexpr int kMaxDeg = 32;     // links per droplet held in the adjacency set
constexpr int kScanBlock = 1024;
constexpr int kCell = 32;       // target edge of a centre-grid cell (nodes): about one droplet spacing
constexpr int kErrDegree = 1;   // a droplet has more than kMaxDeg links
constexpr int kErrDrops = 2;    // more droplets than max_drops
constexpr int kErrUnion = 4;    // a union-find loop ran past its bound
constexpr unsigned kGridCap = 4 * 152;  // blocks of the grid-stride kernels (4 per SM of a GB300)

// Header at the start of the workspace (device-written counts, host-written sizes).
struct Header {
  int n_drops, n_links, err, max_drops;
  int nx, ny, periodic_y, ncx, ncy;
  int pad[7];
};

// A centre as the colouring stages it: the FP64 centre (the oracle's values), its integer parts and
// a two-float split of its fractions.  Written per droplet by centre_final, sorted by cell in cell_fill.
struct alignas(16) CRec {
  double x, y;
  float4 f;  // fraction of x (hi, lo), fraction of y (hi, lo)
  int2 i;    // floor(x), floor(y)
  int id, pad;
};

struct DLayout {
  size_t hdr, lab, did, col, rmask, woff, crec_id, crec, blk, cnt, sx, sy, root, cx, cy, adj, deg, lcount, loff, dblk, ccount, cstart, cfill,
      citems, cblk, links, total;
  long long N;
  int nblk, max_drops, ncx, ncy, ncell, dnblk, cnblk;
  long long max_links;
};

inline DLayout layout(int nx, int ny, int max_drops) {
  DLayout L{};
  L.N = (long long)nx * ny;
  L.max_drops = max_drops;
  L.nblk = (int)((L.N + kScanBlock - 1) / kScanBlock);
  L.dnblk = (max_drops + kScanBlock - 1) / kScanBlock;
  L.ncx = nx / kCell > 0 ? nx / kCell : 1;
  L.ncy = ny / kCell > 0 ? ny / kCell : 1;
  L.ncell = L.ncx * L.ncy;
  L.cnblk = (L.ncell + kScanBlock - 1) / kScanBlock;
  L.max_links = (long long)max_drops * kMaxDeg / 2;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += round_up(bytes, kAlign);
    return o;
  };
  const size_t M = (size_t)max_drops;
  L.hdr = take(sizeof(Header));
  L.lab = take((size_t)L.N * 4);
  L.did = take((size_t)L.N * 4);
  L.col = take((size_t)L.N * 4);
  L.rmask = take((size_t)(L.N + 31) / 32 * 4);
  L.woff = take((size_t)(L.N + 31) / 32 * 4);
  L.blk = take((size_t)(L.nblk + 1) * 4);
  L.cnt = take(M * 8);
  L.sx = take(M * 8);
  L.sy = take(M * 8);
  L.root = take(M * 4);
  L.cx = take(M * 8);
  L.cy = take(M * 8);
  L.adj = take(M * kMaxDeg * 4);
  L.deg = take(M * 4);
  L.lcount = take(M * 4);
  L.loff = take(M * 4);
  L.dblk = take((size_t)(L.dnblk + 1) * 4);
  L.ccount = take((size_t)L.ncell * 4);
  L.cstart = take((size_t)L.ncell * 4);
  L.cfill = take((size_t)L.ncell * 4);
  L.citems = take(M * 4);
  L.crec_id = take(M * sizeof(CRec));
  L.crec = take(M * sizeof(CRec));
  L.cblk = take((size_t)(L.cnblk + 1) * 4);
  L.links = take((size_t)L.max_links * 2 * 4);
  L.total = off;
  return L;
}

// Device view of one workspace.
struct DView {
  Header* hdr;
  int *lab, *did, *col, *blk;
  unsigned* rmask;  // per 32 nodes: the bits of the roots
  int* woff;        // per 32 nodes: the number of roots before them
  unsigned long long* cnt;
  long long *sx, *sy;
  int* root;
  double *cx, *cy;
  int *adj, *deg, *lcount, *loff, *dblk, *ccount, *cstart, *cfill, *citems, *cblk, *links;
  CRec *crec_id, *crec;  // centre records by droplet id, and sorted by cell
};

inline DView view(void* ws, const DLayout& L) {
  unsigned char* b = static_cast<unsigned char*>(ws);
  DView v;
  v.hdr = reinterpret_cast<Header*>(b + L.hdr);
  v.lab = reinterpret_cast<int*>(b + L.lab);
  v.did = reinterpret_cast<int*>(b + L.did);
  v.col = reinterpret_cast<int*>(b + L.col);
  v.rmask = reinterpret_cast<unsigned*>(b + L.rmask);
  v.woff = reinterpret_cast<int*>(b + L.woff);
  v.blk = reinterpret_cast<int*>(b + L.blk);
  v.cnt = reinterpret_cast<unsigned long long*>(b + L.cnt);
  v.sx = reinterpret_cast<long long*>(b + L.sx);
  v.sy = reinterpret_cast<long long*>(b + L.sy);
  v.root = reinterpret_cast<int*>(b + L.root);
  v.cx = reinterpret_cast<double*>(b + L.cx);
  v.cy = reinterpret_cast<double*>(b + L.cy);
  v.adj = reinterpret_cast<int*>(b + L.adj);
  v.deg = reinterpret_cast<int*>(b + L.deg);
  v.lcount = reinterpret_cast<int*>(b + L.lcount);
  v.loff = reinterpret_cast<int*>(b + L.loff);
  v.dblk = reinterpret_cast<int*>(b + L.dblk);
  v.ccount = reinterpret_cast<int*>(b + L.ccount);
  v.cstart = reinterpret_cast<int*>(b + L.cstart);
  v.cfill = reinterpret_cast<int*>(b + L.cfill);
  v.citems = reinterpret_cast<int*>(b + L.citems);
  v.crec_id = reinterpret_cast<CRec*>(b + L.crec_id);
  v.crec = reinterpret_cast<CRec*>(b + L.crec);
  v.cblk = reinterpret_cast<int*>(b + L.cblk);
  v.links = reinterpret_cast<int*>(b + L.links);
  return v;
}

struct Geo {
  int nx, ny, periodic_y;
  const uint8_t* mask;
};

__device__ __forceinline__ bool is_solid(const Geo& g, int x, int y) {
  if (!g.periodic_y && (y == 0 || y == g.ny - 1)) return true;
  return g.mask != nullptr && g.mask[(long long)y * g.nx + x] != 0;
}

// ---------------------------------------------------------------- exclusive scan (3 kernels)

// in[i] for i < n (0 beyond); bsum[b] = sum of block b.
__global__ void scan_block_sums(const int* __restrict__ in, long long n, int* __restrict__ bsum) {
  __shared__ int s_warp[kScanBlock / 32];
  const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  int v = i < n ? in[i] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int w = s_warp[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = w;
  }
}

// Block-wide inclusive scan of one value per thread (kScanBlock threads); *total (may be NULL)
// receives the block total.
__device__ __forceinline__ int block_inclusive_scan(int v, int* s_warp, int* total = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) s_warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const int add = warp > 0 ? s_warp[warp - 1] : 0;
  if (total) *total = s_warp[kScanBlock / 32 - 1];
  __syncthreads();
  return v + add;
}

// One block: exclusive scan of bsum[0 .. nb) in place, bsum[nb] = total.
__global__ void scan_block_offsets(int* __restrict__ bsum, int nb) {
  __shared__ int s_warp[kScanBlock / 32];
  int carry = 0;
  for (int base = 0; base < nb; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    int total = 0;
    const int inc = block_inclusive_scan(v, s_warp, &total);
    if (i < nb) bsum[i] = carry + inc - v;
    carry += total;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

// out[i] = exclusive prefix of in[i] (out may alias in).
__global__ void scan_apply(const int* in, long long n, const int* __restrict__ boff, int* out) {
  __shared__ int s_warp[kScanBlock / 32];
  const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  const int inc = block_inclusive_scan(v, s_warp);
  if (i < n) out[i] = boff[blockIdx.x] + inc - v;
}

cudaError_t exclusive_scan(const int* in, long long n, int* out, int* bsum, cudaStream_t s) {
  const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
  if (nb == 0) return cudaMemsetAsync(bsum, 0, sizeof(int), s);
  scan_block_sums<<<nb, kScanBlock, 0, s>>>(in, n, bsum);
  scan_block_offsets<<<1, kScanBlock, 0, s>>>(bsum, nb);
  scan_apply<<<nb, kScanBlock, 0, s>>>(in, n, bsum, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- labels (D1-D3)
//
// Union-find with every root the smallest node of its set (a hook points the larger root at the
// smaller one), in two levels: each CTA labels a 32 x 32 tile in shared memory (label_local), so
// only the edges that cross a tile border, or the periodic seams, are united in global memory
// (label_border); the parent chains left there run between tile-local roots and stay short.
constexpr int kLT = 32;           // label tile edge
constexpr int kLThreads = 256;

// Root of a, following parents; -1 if the chain is broken or longer than the bound.
__device__ __forceinline__ int find_root(const int* lab, int a, int bound) {
  int r = a;
  for (int k = 0; k < bound; ++k) {
    const int p = lab[r];
    if (p == r) return r;
    if (p < 0) return -1;
    r = p;
  }
  return -1;
}

// Hook the larger root under the smaller one until a and b share a root (lab in global or shared
// memory); false when a loop ran past its bound.
__device__ __forceinline__ bool unite(int* lab, int a, int b, int bound) {
  for (int k = 0; k < bound; ++k) {
    a = find_root(lab, a, bound);
    b = find_root(lab, b, bound);
    if (a < 0 || b < 0) return false;
    if (a == b) return true;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(&lab[a], b);
    if (old == a) return true;  // a was still a root: hooked
    a = old;                    // a was hooked meanwhile; continue from its new parent
  }
  return false;
}

// One CTA per 32 x 32 tile, one warp per row of 32 nodes (a row at a time): D1 foreground and, by a
// warp ballot, the runs of consecutive foreground nodes, each node pointing at its run's first node;
// then one union per overlap of two runs in consecutive rows; then the global index of each node's
// tile-local root (the tile's row-major order is the lattice's order, so the local root, the
// smallest run start of the set, is also its smallest node in global numbering).
__global__ void __launch_bounds__(kLThreads) label_local(const double* __restrict__ rho1, double threshold, Geo g,
                                                         int* __restrict__ lab, int* err) {
  static_assert(kLT == 32, "one lane per tile column");
  __shared__ int s[kLT * kLT];
  __shared__ unsigned s_fg[kLT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = kLThreads / 32;
  const int x0 = blockIdx.x * kLT, y0 = blockIdx.y * kLT, x = x0 + lane;
  constexpr int kRows = kLT / (kLThreads / 32);  // rows per warp, their rho_1 loads issued together
  double v[kRows];
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const int y = y0 + warp + j * nwarp;
    v[j] = (x < g.nx && y < g.ny) ? rho1[y * g.nx + x] : 0.0;
  }
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const int ly = warp + j * nwarp, y = y0 + ly;
    const bool fg = x < g.nx && y < g.ny && !is_solid(g, x, y) && v[j] > threshold;
    const unsigned mask = __ballot_sync(0xffffffffu, fg);
    const unsigned starts = mask & ~(mask << 1);                            // first node of each run
    const int start = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));  // this lane's run (if fg)
    s[ly * kLT + lane] = fg ? ly * kLT + start : -1;
    if (lane == 0) s_fg[ly] = mask;
  }
  __syncthreads();
  bool ok = true;
  for (int ly = warp; ly + 1 < kLT; ly += nwarp) {
    const unsigned both = s_fg[ly] & s_fg[ly + 1];
    if ((both & ~(both << 1)) >> lane & 1u)  // first column of an overlap of a run below and a run above
      ok &= unite(s, ly * kLT + lane, (ly + 1) * kLT + lane, 2 * kLT * kLT);
  }
  if (!ok) atomicOr(err, kErrUnion);
  __syncthreads();
  for (int ly = warp; ly < kLT; ly += nwarp) {
    const int y = y0 + ly;
    if (x >= g.nx || y >= g.ny) continue;
    const int i = ly * kLT + lane;
    int out = -1;
    if (s[i] >= 0) {
      const int r = find_root(s, i, kLT * kLT);
      out = r < 0 ? -1 : (y0 + r / kLT) * g.nx + x0 + (r & (kLT - 1));
    }
    lab[y * g.nx + x] = out;
  }
}

// Unions across tile borders: the right edge of each tile's last column (x + 1 wraps at nx) and the
// upper edge of each tile's last row (y + 1 wraps when periodic_y).  Threads [0, ny * ncol) take the
// vertical borders, the rest the horizontal ones.
__global__ void label_border(Geo g, int ncol, int nrow, int* lab, int* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nv = g.ny * ncol;
  int n, m;
  if (t < nv) {
    const int y = t / ncol, c = t - y * ncol;
    const int x = min(c * kLT + kLT - 1, g.nx - 1);
    n = y * g.nx + x;
    m = y * g.nx + (x + 1 == g.nx ? 0 : x + 1);
  } else if (t < nv + g.nx * nrow) {
    const int u = t - nv, r = u / g.nx, x = u - r * g.nx;
    const int y = min(r * kLT + kLT - 1, g.ny - 1);
    int yu = y + 1;
    if (yu == g.ny) {
      if (!g.periodic_y) return;
      yu = 0;
    }
    n = y * g.nx + x;
    m = yu * g.nx + x;
  } else {
    return;
  }
  if (n == m || lab[n] < 0 || lab[m] < 0) return;
  if (!unite(lab, n, m, 1 << 26)) atomicOr(err, kErrUnion);
}

// Grid-wide node passes that give each thread kPer nodes, n = 1024 b + 256 j + t (j < kPer), issue the
// loads of all of them before using any: one node per thread left each warp waiting on one or two
// dependent loads at a time (at 4096 x 2048: flatten 46 -> 23 us, centre sums 58 -> 46 us).
constexpr int kPassThreads = 256, kPer = kScanBlock / kPassThreads;

// Final labels (the roots), the root bits of every 32 nodes (rmask) and per 1024-node block the number
// of roots (the first pass of the id scan).  The root searches of a thread's nodes advance one parent
// link at a time, together.
__global__ void __launch_bounds__(kPassThreads) label_flatten(int N, int* lab, unsigned* __restrict__ rmask,
                                                             int* __restrict__ bsum, int* err) {
  __shared__ int s_warp[kPassThreads / 32];
  const int base = blockIdx.x * kScanBlock + threadIdx.x;
  int r[kPer];
  bool fg[kPer], live[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int n = base + j * kPassThreads;
    r[j] = n < N ? lab[n] : -1;  // the node's parent (or -1: background or outside)
    fg[j] = r[j] >= 0;
    live[j] = fg[j];
  }
  bool ok = true;
  for (int k = 0; k < (1 << 26); ++k) {  // bounded: a parent chain is shorter than the lattice
    int p[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) p[j] = live[j] ? lab[r[j]] : 0;
    bool any = false;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (!live[j]) continue;
      if (p[j] == r[j]) {
        live[j] = false;  // r[j] is a root
      } else if (p[j] < 0) {
        live[j] = false;  // broken chain
        r[j] = -1;
      } else {
        r[j] = p[j];
        any = true;
      }
    }
    if (!any) break;
    if (k + 1 == (1 << 26)) {
#pragma unroll
      for (int j = 0; j < kPer; ++j)
        if (live[j]) r[j] = -1;
    }
  }
  int count = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int n = base + j * kPassThreads;
    bool root = false;
    if (fg[j]) {
      if (r[j] >= 0) {
        lab[n] = r[j];  // every node of a chain resolves to the same root; concurrent writes store roots only
        root = r[j] == n;
      } else {
        ok = false;
      }
    }
    const unsigned bits = __ballot_sync(0xffffffffu, root);
    if ((threadIdx.x & 31) == 0 && n < N) rmask[n >> 5] = bits;
    count += __popc(bits);
  }
  if (!ok) atomicOr(err, kErrUnion);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = count;
  __syncthreads();
  if (threadIdx.x < 32) {
    int w = threadIdx.x < kPassThreads / 32 ? s_warp[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) bsum[blockIdx.x] = w;
  }
}

// One block: exclusive scan of in[0 .. n) into out (out may alias in); returns the total to every
// thread.
__device__ int block_scan_loop(const int* in, int* out, int n, int* s_warp) {
  int carry = 0;
  for (int base = 0; base < n; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int total = 0;
    const int inc = block_inclusive_scan(v, s_warp, &total);
    if (i < n) out[i] = carry + inc - v;
    carry += total;
  }
  return carry;
}

// One block: exclusive scan of the per-block root counts in place (bsum[nb] = total) and the droplet
// count in the header (clamped to max_drops, kErrDrops beyond).
__global__ void __launch_bounds__(kScanBlock) label_count(int* bsum, int nb, Header* h, int max_drops) {
  __shared__ int s_warp[kScanBlock / 32];
  const int total = block_scan_loop(bsum, bsum, nb, s_warp);
  if (threadIdx.x == 0) {
    bsum[nb] = total;
    h->n_drops = total < max_drops ? total : max_drops;
    if (total > max_drops) atomicOr(&h->err, kErrDrops);
  }
}

// Second pass of the id scan, per 32 nodes: woff[w] = number of roots before node 32 w (the block's
// offset plus a warp scan of the root counts of the block's 32 words).  A root's id (D3) is then
// woff[n / 32] plus the number of roots below it in its word.
__global__ void warp_offsets(int n_words, const unsigned* __restrict__ rmask, const int* __restrict__ boff,
                             int* __restrict__ woff) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;  // blockDim is a multiple of 32: a warp = one scan block
  const int c = w < n_words ? __popc(rmask[w]) : 0;
  int inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if ((threadIdx.x & 31) >= o) inc += t;
  }
  if (w < n_words) woff[w] = boff[w >> 5] + inc - c;
}

__device__ __forceinline__ int root_id(const unsigned* __restrict__ rmask, const int* __restrict__ woff, int r) {
  return woff[r >> 5] + __popc(rmask[r >> 5] & ((1u << (r & 31)) - 1u));
}

// ---------------------------------------------------------------- centres (D4)

__device__ __forceinline__ int min_image_i(int d, int n) {
  if (2 * d > n) d -= n;
  if (2 * d <= -n) d += n;
  return d;
}

// Writes every node's droplet id (did, -1 for background) and the root table (root[id] = the
// droplet's smallest node), and adds each node's offset from that node (minimum image) and a count
// of one to the droplet's sums.  Lanes of a warp mostly see the same droplet: per distinct droplet
// in the warp one 32-bit warp reduction and one 64-bit atomic per sum, so the sums are exact and
// order independent.
__global__ void __launch_bounds__(kPassThreads) centre_sums(Geo g, const int* __restrict__ lab,
                                                           const unsigned* __restrict__ rmask,
                                                           const int* __restrict__ woff,
                                                           const Header* __restrict__ h, int* __restrict__ did,
                                                           int* __restrict__ root, unsigned long long* cnt,
                                                           long long* sx, long long* sy) {
  const int N = g.nx * g.ny;
  const int base = blockIdx.x * kScanBlock + threadIdx.x;
  int l[kPer], d[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int n = base + j * kPassThreads;
    l[j] = n < N ? lab[n] : -1;
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) d[j] = l[j] >= 0 ? root_id(rmask, woff, l[j]) : -1;
  const int n_drops = h->n_drops;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int n = base + j * kPassThreads;
    if (n < N) did[n] = d[j];
    const bool mine = d[j] >= 0 && d[j] < n_drops;
    if (mine && l[j] == n) root[d[j]] = n;
    int dx = 0, dy = 0;
    if (mine) {
      const int x = n % g.nx, y = n / g.nx, rx = l[j] % g.nx, ry = l[j] / g.nx;
      dx = min_image_i(x - rx, g.nx);
      dy = g.periodic_y ? min_image_i(y - ry, g.ny) : (y - ry);
    }
    const unsigned active = __ballot_sync(0xffffffffu, mine);
    if (!mine) continue;
    unsigned rest = active;
    while (rest) {  // one iteration per distinct droplet among the active lanes (at most 32)
      const int dl = __shfl_sync(active, d[j], __ffs(rest) - 1);
      const bool in_group = d[j] == dl;
      const unsigned group = __ballot_sync(active, in_group);
      const int gx = __reduce_add_sync(active, in_group ? dx : 0);
      const int gy = __reduce_add_sync(active, in_group ? dy : 0);
      if ((int)(threadIdx.x & 31) == __ffs(group) - 1) {
        atomicAdd(cnt + dl, (unsigned long long)__popc(group));
        atomicAdd(reinterpret_cast<unsigned long long*>(sx + dl), (unsigned long long)(long long)gx);
        atomicAdd(reinterpret_cast<unsigned long long*>(sy + dl), (unsigned long long)(long long)gy);
      }
      rest &= ~group;
    }
  }
}

// Per droplet (grid-stride over the count in the header): the centre, wrapped into the lattice, and
// its cell of the centre grid (kept in dcell) with the cell's count.
__global__ void centre_final(Geo g, const Header* __restrict__ h, const int* __restrict__ root,
                             const unsigned long long* __restrict__ cnt, const long long* __restrict__ sx,
                             const long long* __restrict__ sy, double* cx, double* cy, int ncx, int ncy,
                             int* __restrict__ ccount, int* __restrict__ dcell, CRec* __restrict__ rec) {
  const int n_drops = h->n_drops;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n_drops; d += gridDim.x * blockDim.x) {
    const int r = root[d];
    const double rx = (double)(r % g.nx), ry = (double)(r / g.nx);
    double x = __dadd_rn(rx, __ddiv_rn((double)sx[d], (double)cnt[d]));
    double y = __dadd_rn(ry, __ddiv_rn((double)sy[d], (double)cnt[d]));
    if (x < 0.0) x = __dadd_rn(x, (double)g.nx);
    else if (x >= (double)g.nx) x = __dsub_rn(x, (double)g.nx);
    if (g.periodic_y) {
      if (y < 0.0) y = __dadd_rn(y, (double)g.ny);
      else if (y >= (double)g.ny) y = __dsub_rn(y, (double)g.ny);
    }
    cx[d] = x;
    cy[d] = y;
    CRec cr;
    cr.x = x;
    cr.y = y;
    const double fx0 = floor(x), fy0 = floor(y);
    const double fx = __dsub_rn(x, fx0), fy = __dsub_rn(y, fy0);  // exact: a number and its floor are within one
    const float fxh = __double2float_rn(fx), fyh = __double2float_rn(fy);
    cr.f = make_float4(fxh, __double2float_rn(__dsub_rn(fx, (double)fxh)), fyh,
                       __double2float_rn(__dsub_rn(fy, (double)fyh)));
    cr.i = make_int2((int)fx0, (int)fy0);
    cr.id = d;
    cr.pad = 0;
    rec[d] = cr;
    // cell of the centre: equal-width cells, nx / ncx by ny / ncy
    int ix = (int)(x * ncx / g.nx), iy = (int)(y * ncy / g.ny);
    ix = ix < 0 ? 0 : (ix >= ncx ? ncx - 1 : ix);
    iy = iy < 0 ? 0 : (iy >= ncy ? ncy - 1 : iy);
    const int c = iy * ncx + ix;
    dcell[d] = c;
    atomicAdd(ccount + c, 1);
  }
}

// One block: cell starts (exclusive scan of the counts).
__global__ void __launch_bounds__(kScanBlock) cell_scan(int ncell, const int* __restrict__ ccount,
                                                       int* __restrict__ cstart) {
  __shared__ int s_warp[kScanBlock / 32];
  block_scan_loop(ccount, cstart, ncell, s_warp);
}

// Per droplet (grid-stride over the count in the header): its slot in its cell's list of droplet ids,
// and its centre record at the same slot.
__global__ void cell_fill(const Header* __restrict__ h, const int* __restrict__ cstart,
                          const int* __restrict__ dcell, int* cfill, int* __restrict__ citems,
                          const CRec* __restrict__ rec_id, CRec* __restrict__ rec) {
  const int n_drops = h->n_drops;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n_drops; d += gridDim.x * blockDim.x) {
    const int c = dcell[d];
    const int at = cstart[c] + atomicAdd(cfill + c, 1);
    citems[at] = d;
    rec[at] = rec_id[d];
  }
}

// ---------------------------------------------------------------- nearest centre (D5)

struct Grid {
  const double *cx, *cy;
  const int *cstart, *ccount, *citems;
  int ncx, ncy;
  double cw_min;  // smaller cell edge
  double cw2_d;   // (2 cw_min)^2 (1 - 1e-9): a staged nearest distance below it is exact
  float cw2_f;    // cw2_d rounded down to FP32
};

// Nearest centre to (x, y): rings of cells around the point's cell until no unvisited cell can hold a
// closer centre.  A cell at ring distance >= r + 1 lies >= r cell edges away in x or y, so after ring
// r every centre not yet seen is farther than (r - 1) * cw_min (one ring of margin for the rounding
// of the cell index).  Ties keep the smaller id.
__device__ int nearest_centre(const Geo& g, const Grid& G, double x, double y, double* best_out) {
  const double hx = 0.5 * g.nx, hy = 0.5 * g.ny;
  int ix = (int)(x * G.ncx / g.nx), iy = (int)(y * G.ncy / g.ny);
  ix = ix < 0 ? 0 : (ix >= G.ncx ? G.ncx - 1 : ix);
  iy = iy < 0 ? 0 : (iy >= G.ncy ? G.ncy - 1 : iy);
  double best = 0.0;
  int best_id = -1;
  const int rmax = (G.ncx > G.ncy ? G.ncx : G.ncy) + 1;
  for (int r = 0; r <= rmax; ++r) {
    for (int jy = iy - r; jy <= iy + r; ++jy) {
      int cyi = jy;
      if (g.periodic_y) cyi = ((jy % G.ncy) + G.ncy) % G.ncy;
      else if (jy < 0 || jy >= G.ncy) continue;
      const bool edge_row = (jy == iy - r) || (jy == iy + r);
      for (int jx = ix - r; jx <= ix + r; jx += (edge_row || r == 0) ? 1 : 2 * r) {
        const int cxi = ((jx % G.ncx) + G.ncx) % G.ncx;
        const int c = cyi * G.ncx + cxi;
        const int s = G.cstart[c], e = s + G.ccount[c];
        for (int k = s; k < e; ++k) {
          const int d = G.citems[k];
          double dx = __dsub_rn(x, G.cx[d]);
          if (dx > hx) dx = __dsub_rn(dx, (double)g.nx);
          else if (dx < -hx) dx = __dadd_rn(dx, (double)g.nx);
          double dy = __dsub_rn(y, G.cy[d]);
          if (g.periodic_y) {
            if (dy > hy) dy = __dsub_rn(dy, (double)g.ny);
            else if (dy < -hy) dy = __dadd_rn(dy, (double)g.ny);
          }
          const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
          if (best_id < 0 || d2 < best || (d2 == best && d < best_id)) {
            best = d2;
            best_id = d;
          }
        }
      }
    }
    if (best_id >= 0 && r >= 1) {
      const double bound = (double)(r - 1) * G.cw_min;
      if (best < bound * bound) break;
    }
  }
  if (best_out) *best_out = best;
  return best_id;
}

// ---------------------------------------------------------------- colours and links (D5, D6)

// Nearest centre: distances screened in FP32.  The node's integer offset from a centre's integer part
// is exact; the minimum image is decided on the offset less the fraction's high part (as the oracle
// decides it on its offset; a decision that differs within an ulp of +-n/2 changes |dx| by an ulp),
// and the offset is recomputed from the wrapped integer, so each screened component is within two
// FP32 roundings of the exact offset and a screened squared distance within 5e-7 (relative) of the
// FP64 one (the oracle's unfused dx*dx + dy*dy).  When every other candidate screens above
// 1.00001 x the best + 1e-3, the best is the strict FP64 minimum and is taken as it is; otherwise (a
// node within that margin of a Voronoi edge) the candidates inside the margin are compared in FP64
// with the oracle's arithmetic and tie rule.  FP64 runs at 1/64 of the FP32 rate on this part, so
// the screen decides almost every node without it.
//
// Staging: a node's centre is looked for among the records of the cells within 2 cells of the node's
// cell (x periodic; y periodic or clipped).  Any centre not staged sits in a cell 3 or more cells from
// the node's cell in x or y, so with two whole cells in between it lies more than 2 cell edges away
// (less about 1e-12 where the FP64 cell index of a centre on a cell boundary rounds up; the 1e-9
// factor of cw2_d covers it): a node whose best staged distance is below 2 cell edges has its exact
// answer; otherwise (and when the staging list overflows) it runs the full ring search.  The staged list is first cut to the centres that can be nearest to a
// node of the group: the centre nearest to the group's middle bounds every node's nearest distance
// by U (its distance + the half-extent of the group), and a centre farther than U from the group's
// box is nobody's nearest (nor tied).  FP32 with margins far above its rounding (1e-4 relative, 1e-2
// absolute) keeps U an upper bound.
constexpr int kVTX = 32, kVTY = 8, kVThreads = kVTX * kVTY;

// Colours with one warp per row of 32 nodes (8 rows a CTA) and no CTA barrier: each warp stages the
// records of the cells within 2 cells of its row's cells (lane = cell, a warp scan places them), cuts
// them to the centres within U of its row, and screens them for its 32 nodes; only __syncwarp orders
// the steps.  The eight warps of a CTA stage overlapping cells (the repeats hit L1).  A 32 x 8 tile
// staged once by the CTA, with CTA barriers between staging, cut and screen, measured 2% slower.
constexpr int kWList = 64;  // staged records per warp; more falls back to the ring search

__global__ void __launch_bounds__(kVThreads) voronoi_rows(Geo g, Grid G, const CRec* __restrict__ rec,
                                                          const Header* __restrict__ h, int* __restrict__ col) {
  __shared__ CRec s_r[kVTY][kWList];
  __shared__ int s_k[kVTY][kWList];  // indices of the kept records
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int n_drops = h->n_drops;
  const int x0 = blockIdx.x * kVTX, y = blockIdx.y * kVTY + wy;
  if (y >= g.ny) return;  // a whole warp: no later warp-wide operation misses a lane
  const int w = min(kVTX, g.nx - x0);
  CRec* const sr = s_r[wy];
  int* const sk = s_k[wy];
  // the warp's cells: x range widened by 2 cells (a window wider than the grid takes each cell once),
  // rows cy - 2 .. cy + 2 (periodic, or clipped)
  const int cxa = (int)((long long)x0 * G.ncx / g.nx) - 2, cxb = (int)((long long)(x0 + w - 1) * G.ncx / g.nx) + 2;
  const int cyc = (int)((long long)y * G.ncy / g.ny);
  const int span = min(cxb - cxa + 1, G.ncx);
  const int rows = g.periodic_y ? min(5, G.ncy) : 5;
  const int ry0 = g.periodic_y && rows < 5 ? 0 : cyc - 2;
  const int ncell = span * rows;
  int start = 0, cnt = 0;
  if (lane < ncell && n_drops > 0) {
    const int r = lane / span, cxi = ((cxa + lane - r * span) % G.ncx + G.ncx) % G.ncx;
    int cyi = ry0 + r;
    bool ok = true;
    if (g.periodic_y) cyi = (cyi % G.ncy + G.ncy) % G.ncy;
    else ok = cyi >= 0 && cyi < G.ncy;
    if (ok) {
      const int cell = cyi * G.ncx + cxi;
      start = G.cstart[cell];
      cnt = G.ccount[cell];
    }
  }
  int off = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, off, o);
    if (lane >= o) off += t;
  }
  const int total = __shfl_sync(0xffffffffu, off, 31);
  off -= cnt;
  const bool staged = n_drops > 0 && ncell <= 32 && total <= kWList;
  int m = 0;
  if (staged && total > 0) {
    for (int k = 0; k < cnt; ++k) sr[off + k] = rec[start + k];
    __syncwarp();
    const float hw = 0.5f * (float)(w - 1);
    const float tcx = (float)x0 + hw, tcy = (float)y;
    auto offset = [&](const CRec& r, float& ax, float& ay) {  // |centre - row middle|, minimum image
      float dx = ((float)r.i.x - tcx) + r.f.x, dy = ((float)r.i.y - tcy) + r.f.z;
      if (dx > 0.5f * g.nx) dx -= (float)g.nx;
      else if (dx < -0.5f * g.nx) dx += (float)g.nx;
      if (g.periodic_y) {
        if (dy > 0.5f * g.ny) dy -= (float)g.ny;
        else if (dy < -0.5f * g.ny) dy += (float)g.ny;
      }
      ax = fabsf(dx);
      ay = fabsf(dy);
    };
    float a0x = 3.0e38f, a0y = 0.0f, a1x = 3.0e38f, a1y = 0.0f, dmin = 3.0e38f;
    if (lane < total) {
      offset(sr[lane], a0x, a0y);
      dmin = a0x * a0x + a0y * a0y;
    }
    if (lane + 32 < total) {
      offset(sr[lane + 32], a1x, a1y);
      dmin = fminf(dmin, a1x * a1x + a1y * a1y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    const float U = (sqrtf(dmin) + hw) * 1.0001f + 0.01f;
    const float e0 = fmaxf(a0x - hw, 0.0f), e1 = fmaxf(a1x - hw, 0.0f);
    const bool k0 = lane < total && e0 * e0 + a0y * a0y <= U * U;
    const bool k1 = lane + 32 < total && e1 * e1 + a1y * a1y <= U * U;
    const unsigned b0 = __ballot_sync(0xffffffffu, k0), b1 = __ballot_sync(0xffffffffu, k1);
    const unsigned below = (1u << lane) - 1u;
    if (k0) sk[__popc(b0 & below)] = lane;
    if (k1) sk[__popc(b0) + __popc(b1 & below)] = lane + 32;
    m = __popc(b0) + __popc(b1);
    __syncwarp();
  }
  const int x = x0 + lane;
  if (lane >= w) return;
  const int n = y * g.nx + x;
  if (is_solid(g, x, y) || n_drops == 0) {
    col[n] = -1;
    return;
  }
  const float fhx = 0.5f * g.nx, fhy = 0.5f * g.ny;
  auto screen = [&](const CRec& r) {
    const int dxi = x - r.i.x, dyi = y - r.i.y;
    float dx = (float)dxi - r.f.x;
    if (dx > fhx) dx = (float)(dxi - g.nx) - r.f.x;
    else if (dx < -fhx) dx = (float)(dxi + g.nx) - r.f.x;
    dx -= r.f.y;
    float dy = (float)dyi - r.f.z;
    if (g.periodic_y) {
      if (dy > fhy) dy = (float)(dyi - g.ny) - r.f.z;
      else if (dy < -fhy) dy = (float)(dyi + g.ny) - r.f.z;
    }
    dy -= r.f.w;
    return dx * dx + dy * dy;
  };
  int best_id = -1;
  bool settled = false;
  if (staged && m > 0) {
    float b1 = 3.0e38f, b2 = 3.0e38f;
    int k1 = -1;
    for (int k = 0; k < m; ++k) {
      const float d2 = screen(sr[sk[k]]);
      if (d2 < b1) {
        b2 = b1;
        b1 = d2;
        k1 = k;
      } else if (d2 < b2) {
        b2 = d2;
      }
    }
    const float keep = b1 * 1.00001f + 1e-3f;
    if (b2 > keep) {
      best_id = sr[sk[k1]].id;
      settled = keep < G.cw2_f;
    } else {
      const double px = (double)x, py = (double)y, hx = 0.5 * g.nx, hy = 0.5 * g.ny;
      double best = 0.0;
      for (int kk = 0; kk < m; ++kk) {
        const CRec& r = sr[sk[kk]];
        if (screen(r) > keep) continue;
        double dx = __dsub_rn(px, r.x);
        if (dx > hx) dx = __dsub_rn(dx, (double)g.nx);
        else if (dx < -hx) dx = __dadd_rn(dx, (double)g.nx);
        double dy = __dsub_rn(py, r.y);
        if (g.periodic_y) {
          if (dy > hy) dy = __dsub_rn(dy, (double)g.ny);
          else if (dy < -hy) dy = __dadd_rn(dy, (double)g.ny);
        }
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        if (best_id < 0 || d2 < best || (d2 == best && r.id < best_id)) {
          best = d2;
          best_id = r.id;
        }
      }
      settled = best_id >= 0 && best < G.cw2_d;
    }
  }
  if (!settled) best_id = nearest_centre(g, G, (double)x, (double)y, nullptr);
  col[n] = best_id;
}

// Inserts b into a's adjacency set unless it is there: the set is read first and the first empty
// slot claimed with one compare-and-swap (re-read when another insert took it), so an insert costs
// one atomic when it does not race.
__device__ __forceinline__ void adj_insert(int* adj, int* deg, int a, int b, int* err) {
  int* slots = adj + (long long)a * kMaxDeg;
  int k = 0;
  while (k < kMaxDeg) {
    const int v = *reinterpret_cast<volatile int*>(slots + k);
    if (v == b) return;
    if (v != -1) {
      ++k;
      continue;
    }
    const int old = atomicCAS(slots + k, -1, b);
    if (old == -1) {
      atomicAdd(deg + a, 1);
      return;
    }
    if (old == b) return;
    ++k;  // the slot was taken meanwhile by another value: the next one
  }
  atomicOr(err, kErrDegree);
}

// Links (D6) of the 2 x 2 window whose lower-left corner is node n (corners in cyclic order 00, 10, 11,
// 01), one window per thread: few windows hold three or four colours, and each of those runs its
// inserts one after another (four windows per thread measured 1.5-2x slower).
__global__ void voronoi_links(Geo g, const int* __restrict__ col, int* adj, int* deg, int* err) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;  // one block row per lattice row
  if (x >= g.nx) return;
  if (!g.periodic_y && y == g.ny - 1) return;
  const int x1 = x + 1 == g.nx ? 0 : x + 1, y1 = y + 1 == g.ny ? 0 : y + 1;
  const int c[4] = {col[y * g.nx + x], col[y * g.nx + x1], col[y1 * g.nx + x1], col[y1 * g.nx + x]};
  if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[3] < 0) return;
  if (c[0] == c[1] && c[1] == c[2] && c[2] == c[3]) return;
  int dist[4], k = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    bool seen = false;
    for (int j = 0; j < k; ++j) seen |= dist[j] == c[i];
    if (!seen) dist[k++] = c[i];
  }
  if (k == 3) {
    const int p[3][2] = {{dist[0], dist[1]}, {dist[1], dist[2]}, {dist[0], dist[2]}};
    for (int i = 0; i < 3; ++i) {
      adj_insert(adj, deg, p[i][0], p[i][1], err);
      adj_insert(adj, deg, p[i][1], p[i][0], err);
    }
  } else if (k == 4) {
    for (int i = 0; i < 4; ++i) {
      const int a = c[i], b = c[(i + 1) & 3];
      adj_insert(adj, deg, a, b, err);
      adj_insert(adj, deg, b, a, err);
    }
  }
}

// One warp per droplet (grid-stride over the count in the header): sorts the adjacency set
// ascending in registers (bitonic network over the 32 slots, empty slots last) and counts the links
// to larger ids.  The filled slots of a set are a prefix (an insert takes the first empty slot).
__global__ void adj_sort(const Header* __restrict__ h, int* adj, const int* __restrict__ deg,
                         int* __restrict__ lcount) {
  static_assert(kMaxDeg == 32, "one adjacency slot per lane");
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int n_drops = h->n_drops;
  for (int d = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); d < n_drops; d += warps) {
    int* a = adj + (size_t)d * kMaxDeg;
    const int m = deg[d] < kMaxDeg ? deg[d] : kMaxDeg;
    int v = lane < m ? a[lane] : 0x7fffffff;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int o = __shfl_xor_sync(0xffffffffu, v, j);
        const bool up = (lane & k) == 0, low = (lane & j) == 0;
        v = (low == up) ? min(v, o) : max(v, o);
      }
    }
    if (lane < m) a[lane] = v;
    const unsigned larger = __ballot_sync(0xffffffffu, lane < m && v > d);
    if (lane == 0) lcount[d] = __popc(larger);
  }
}

// One block: link offsets (exclusive scan of the per-droplet counts) and the link count in the header.
__global__ void __launch_bounds__(kScanBlock) links_count(Header* h, const int* __restrict__ lcount,
                                                         int* __restrict__ loff) {
  __shared__ int s_warp[kScanBlock / 32];
  const int total = block_scan_loop(lcount, loff, h->n_drops, s_warp);
  if (threadIdx.x == 0) h->n_links = total;
}

// Per droplet d (grid-stride): its links (d, b) with b > d, ascending, at its offset (at most
// max_links in all; only an adjacency overflow, reported as kErrDegree, can reach that bound).
__global__ void links_write(const Header* __restrict__ h, const int* __restrict__ adj, const int* __restrict__ deg,
                            const int* __restrict__ loff, int* __restrict__ links, long long max_links) {
  const int n_drops = h->n_drops;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < n_drops; d += gridDim.x * blockDim.x) {
    const int* a = adj + (size_t)d * kMaxDeg;
    const int m = deg[d] < kMaxDeg ? deg[d] : kMaxDeg;
    int o = loff[d];
    for (int i = 0; i < m; ++i) {
      const int b = a[i];
      if (b > d && o < max_links) {
        links[2 * o] = d;
        links[2 * o + 1] = b;
        ++o;
      }
    }
  }
}

// Resets one analysis: the header (sizes, zero counts and error bits) and every per-droplet and
// per-cell accumulator the pipeline adds into (grid-stride over the largest of them).
__global__ void drop_reset(Header* h, Header init, unsigned long long* cnt, long long* sx, long long* sy, int* adj,
                           int* deg, int* ccount, int* cfill, int ncell) {
  const int M = init.max_drops;
  const long long total = (long long)M * kMaxDeg > ncell ? (long long)M * kMaxDeg : ncell;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < (long long)M * kMaxDeg) adj[i] = -1;
    if (i < M) {
      cnt[i] = 0;
      sx[i] = 0;
      sy[i] = 0;
      deg[i] = 0;
    }
    if (i < ncell) {
      ccount[i] = 0;
      cfill[i] = 0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *h = init;
}

// ---------------------------------------------------------------- T1 comparison

__device__ __forceinline__ bool has_link(const int* adj, const int* deg, int a, int b) {
  const int* s = adj + (long long)a * kMaxDeg;
  const int m = deg[a] < kMaxDeg ? deg[a] : kMaxDeg;
  for (int i = 0; i < m; ++i)
    if (s[i] == b) return true;
  return false;
}

// match[j] = i when droplet j of `from` and droplet i of `to` are each other's nearest centre
// within d_max; one pass per direction (near[] holds the one-directional nearest).
__global__ void nearest_other(Geo g, Grid to, int n_from, const double* __restrict__ fx, const double* __restrict__ fy,
                              double d2max, int* __restrict__ near) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_from) return;
  double best = 0.0;
  const int i = nearest_centre(g, to, fx[j], fy[j], &best);
  near[j] = (i >= 0 && best <= d2max) ? i : -1;
}

__global__ void mutual(int n_now, const int* __restrict__ near_np, const int* __restrict__ near_pn,
                       int* __restrict__ n2p) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_now) return;
  const int i = near_np[j];
  n2p[j] = (i >= 0 && near_pn[i] == j) ? i : -1;
}

__global__ void invert(int n_now, const int* __restrict__ n2p, int* __restrict__ p2n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_now) return;
  if (n2p[j] >= 0) p2n[n2p[j]] = j;
}

// mode 0: broken links of prev (per prev droplet a, links a < b); mode 1: arising links (per now
// droplet c, links c < d, written in prev ids).  count pass (out == nullptr) and write pass.
__global__ void link_changes(int mode, int n, const int* __restrict__ adj_self, const int* __restrict__ deg_self,
                             const int* __restrict__ adj_other, const int* __restrict__ deg_other,
                             const int* __restrict__ map, const int* __restrict__ cnt_off, int* __restrict__ counts,
                             int* __restrict__ out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  const int* s = adj_self + (long long)a * kMaxDeg;
  const int m = deg_self[a] < kMaxDeg ? deg_self[a] : kMaxDeg;
  int c = 0, o = out ? cnt_off[a] : 0;
  for (int i = 0; i < m; ++i) {
    const int b = s[i];
    if (b <= a) continue;
    const int ma = map[a], mb = map[b];
    if (ma < 0 || mb < 0) continue;
    if (has_link(adj_other, deg_other, ma, mb)) continue;
    if (out) {
      const int lo = mode == 0 ? a : (ma < mb ? ma : mb), hi = mode == 0 ? b : (ma < mb ? mb : ma);
      out[2 * (o + c)] = lo;
      out[2 * (o + c) + 1] = hi;
    }
    ++c;
  }
  if (!out) counts[a] = c;
}

// T1 events: per broken link (a, b), the pairs (c, d) of common prev neighbours of a and b that are
// not linked in prev but are linked now (both matched).
__global__ void t1_events(int n_broken, const int* __restrict__ broken, const int* __restrict__ adj_p,
                          const int* __restrict__ deg_p, const int* __restrict__ adj_n, const int* __restrict__ deg_n,
                          const int* __restrict__ p2n, const int* __restrict__ cnt_off, int* __restrict__ counts,
                          int* __restrict__ out, long long out_cap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_broken) return;
  const int a = broken[2 * k], b = broken[2 * k + 1];
  const int* sa = adj_p + (long long)a * kMaxDeg;
  const int ma = deg_p[a] < kMaxDeg ? deg_p[a] : kMaxDeg;
  int cnt = 0, o = out ? cnt_off[k] : 0;
  for (int i = 0; i < ma; ++i) {
    const int c = sa[i];
    if (!has_link(adj_p, deg_p, b, c)) continue;
    for (int j = i + 1; j < ma; ++j) {
      const int d = sa[j];
      if (!has_link(adj_p, deg_p, b, d) || has_link(adj_p, deg_p, c, d)) continue;
      const int nc = p2n[c], nd = p2n[d];
      if (nc < 0 || nd < 0 || !has_link(adj_n, deg_n, nc, nd)) continue;
      if (out && o + cnt < out_cap) {  // out holds out_cap quadruples
        out[4 * (o + cnt)] = a;
        out[4 * (o + cnt) + 1] = b;
        out[4 * (o + cnt) + 2] = c < d ? c : d;
        out[4 * (o + cnt) + 3] = c < d ? d : c;
      }
      ++cnt;
    }
  }
  if (!out) counts[k] = cnt;
}

// Droplet Nusselt number (Eq. NuDrops) at the node nearest to each centre (x rounded half up,
// periodic; y rounded half up and clamped): (u_y T - kappa dT/dy) / (kappa Delta T / H), dT/dy central
// with the mirror 2 T_w - T at a solid neighbour.  Unfused double arithmetic in the oracle's order.
// NaN when the nearest node is solid.  fields: 5 planes rho1, rho2, T, ux, uy of nx * ny doubles.
__global__ void droplet_nusselt(Geo g, int n_drops, const double* __restrict__ cx, const double* __restrict__ cy,
                                const double* __restrict__ fields, double kappa, double den, double T_down,
                                double T_up, double* __restrict__ nu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_drops) return;
  const long long N = (long long)g.nx * g.ny;
  int x = (int)floor(__dadd_rn(cx[i], 0.5)) % g.nx;
  int y = (int)floor(__dadd_rn(cy[i], 0.5));
  y = y < 0 ? 0 : (y > g.ny - 1 ? g.ny - 1 : y);
  if (is_solid(g, x, y)) {
    nu[i] = __longlong_as_double(0x7ff8000000000000ll);  // quiet NaN
    return;
  }
  const double* T = fields + 2 * N;
  const double* uy = fields + 4 * N;
  const long long n = (long long)y * g.nx + x;
  const double t = T[n];
  auto neighbour = [&](int yy) {
    if (g.periodic_y) yy = (yy + g.ny) % g.ny;
    if (is_solid(g, x, yy)) {
      const double tw = (2 * yy < g.ny) ? T_down : T_up;
      return __dsub_rn(__dmul_rn(2.0, tw), t);
    }
    return T[(long long)yy * g.nx + x];
  };
  const double dTdy = __dmul_rn(0.5, __dsub_rn(neighbour(y + 1), neighbour(y - 1)));
  nu[i] = __ddiv_rn(__dsub_rn(__dmul_rn(uy[n], t), __dmul_rn(kappa, dTdy)), den);
}

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace drops
}  // namespace tlb

using namespace tlb;
using namespace tlb::drops;

namespace {

int dfail(lb_handle* h, int code, const char* msg, cudaError_t e = cudaSuccess) {
  if (h)
    std::snprintf(h->err, sizeof h->err, "%s%s%s", msg, e != cudaSuccess ? ": " : "",
                  e != cudaSuccess ? cudaGetErrorString(e) : "");
  return code;
}

cudaError_t fields_into(const lb_handle* h, double* stage) {
  const int pr = h->p.precision;
  if (pr == LB_DF64) return launch_df64(MODE_FIELDS, h->cfg, h->buf[h->cur], nullptr, stage, h->stream);
  return pr == LB_FP64 ? launch_f64(MODE_FIELDS, h->cfg, h->buf[h->cur], nullptr, stage, h->stream)
                       : (pr == LB_FP32_SHIFTED ? launch_f32(MODE_FIELDS, h->cfg, h->buf[h->cur], nullptr, stage, h->stream)
                                                : launch_f32h(MODE_FIELDS, h->cfg, h->buf[h->cur], nullptr, stage, h->stream));
}

Grid grid_of(const DView& v, const DLayout& L, const lb_params& p) {
  Grid G;
  G.cx = v.cx;
  G.cy = v.cy;
  G.cstart = v.cstart;
  G.ccount = v.ccount;
  G.citems = v.citems;
  G.ncx = L.ncx;
  G.ncy = L.ncy;
  const double wx = (double)p.nx / L.ncx, wy = (double)p.ny / L.ncy;
  G.cw_min = wx < wy ? wx : wy;
  G.cw2_d = 4.0 * G.cw_min * G.cw_min * (1.0 - 1e-9);
  G.cw2_f = (float)G.cw2_d;
  if ((double)G.cw2_f > G.cw2_d) G.cw2_f = std::nextafter(G.cw2_f, 0.0f);
  return G;
}

bool check_ws(const lb_handle* h, const void* ws, size_t bytes, int max_drops, DLayout* L) {
  if (!ws || ((uintptr_t)ws % kAlign) != 0 || max_drops < 1) return false;
  *L = layout(h->p.nx, h->p.ny, max_drops);
  return bytes >= L->total;
}

int read_header(lb_handle* h, const void* ws, Header* out) {
  const cudaError_t e = cudaMemcpyAsync(out, ws, sizeof(Header), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return dfail(h, LB_ECUDA, "droplet header", e);
  const cudaError_t e2 = cudaStreamSynchronize(h->stream);
  if (e2 != cudaSuccess) return dfail(h, LB_ECUDA, "droplet header", e2);
  return LB_OK;
}

// Enqueues one droplet analysis of the current state on stream s (no host synchronisation).
cudaError_t enqueue_analysis(const lb_handle* h, const DView& v, const DLayout& L, const Header& hdr, double threshold,
                             int max_drops, cudaStream_t s) {
  const Geo g{h->p.nx, h->p.ny, h->p.periodic_y, h->cfg.mask};
  double* stage = static_cast<double*>(h->buf[h->cur ^ 1]);  // rho1 is plane 0 of the fields
  const int N = (int)L.N;  // nx * ny fits in 31 bits (lb_init)
  const int T = 256;
  // the per-droplet kernels run grid-stride over the count the labelling writes into the header
  auto capped = [](unsigned blocks) { return blocks < kGridCap ? blocks : kGridCap; };
  const unsigned per_drop = capped(nb(max_drops, T)), per_drop_warps = capped(nb((long long)max_drops * 32, T));
  const unsigned reset_blocks =
      capped(nb((long long)max_drops * kMaxDeg > L.ncell ? (long long)max_drops * kMaxDeg : L.ncell, T));
  int* err = &v.hdr->err;
  cudaError_t e = launch_mode(h->p.precision, MODE_RHO1, h->cfg, h->buf[h->cur], nullptr, stage, s);
  if (e != cudaSuccess) return e;
  drop_reset<<<reset_blocks, T, 0, s>>>(v.hdr, hdr, v.cnt, v.sx, v.sy, v.adj, v.deg, v.ccount, v.cfill, L.ncell);
  // labels (D1-D3): tile-local union-find, unions across tile borders, roots and their ids
  const int ncol = (h->p.nx + kLT - 1) / kLT, nrow = (h->p.ny + kLT - 1) / kLT;
  label_local<<<dim3((unsigned)ncol, (unsigned)nrow), kLThreads, 0, s>>>(stage, threshold, g, v.lab, err);
  label_border<<<nb((long long)h->p.ny * ncol + (long long)h->p.nx * nrow, T), T, 0, s>>>(g, ncol, nrow, v.lab, err);
  label_flatten<<<L.nblk, kPassThreads, 0, s>>>(N, v.lab, v.rmask, v.blk, err);
  label_count<<<1, kScanBlock, 0, s>>>(v.blk, L.nblk, v.hdr, max_drops);
  const int n_words = (N + 31) / 32;
  warp_offsets<<<nb(n_words, T), T, 0, s>>>(n_words, v.rmask, v.blk, v.woff);
  // centres (D4) and the cell grid of the centres
  centre_sums<<<L.nblk, kPassThreads, 0, s>>>(g, v.lab, v.rmask, v.woff, v.hdr, v.did, v.root, v.cnt, v.sx, v.sy);
  centre_final<<<per_drop, T, 0, s>>>(g, v.hdr, v.root, v.cnt, v.sx, v.sy, v.cx, v.cy, L.ncx, L.ncy, v.ccount, v.lcount,
                                      v.crec_id);
  cell_scan<<<1, kScanBlock, 0, s>>>(L.ncell, v.ccount, v.cstart);
  cell_fill<<<per_drop, T, 0, s>>>(v.hdr, v.cstart, v.lcount, v.cfill, v.citems, v.crec_id, v.crec);
  // colours (D5) and links (D6)
  const Grid G = grid_of(v, L, h->p);
  voronoi_rows<<<dim3((unsigned)((h->p.nx + kVTX - 1) / kVTX), (unsigned)((h->p.ny + kVTY - 1) / kVTY)),
                 dim3(kVTX, kVTY), 0, s>>>(g, G, v.crec, v.hdr, v.col);
  voronoi_links<<<dim3(nb(h->p.nx, T), (unsigned)h->p.ny), T, 0, s>>>(g, v.col, v.adj, v.deg, err);
  adj_sort<<<per_drop_warps, T, 0, s>>>(v.hdr, v.adj, v.deg, v.lcount);
  links_count<<<1, kScanBlock, 0, s>>>(v.hdr, v.lcount, v.loff);
  links_write<<<per_drop, T, 0, s>>>(v.hdr, v.adj, v.deg, v.loff, v.links, L.max_links);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int lb_droplets_workspace_size(const lb_handle* h, int max_drops, size_t* bytes) {
  if (!h || !bytes || max_drops < 1) return LB_EINVAL;
  *bytes = layout(h->p.nx, h->p.ny, max_drops).total;
  return LB_OK;
}

int lb_droplets(lb_handle* h, double threshold, int max_drops, void* d_ws, size_t ws_bytes, int* n_drops,
                int* n_links) {
  if (!h) return LB_EINVAL;
  DLayout L;
  if (!check_ws(h, d_ws, ws_bytes, max_drops, &L))
    return dfail(h, LB_ENOSPACE, "droplet workspace too small, misaligned or max_drops < 1");
  if (!(threshold == threshold)) return dfail(h, LB_EINVAL, "threshold is NaN");
  const DView v = view(d_ws, L);
  Header hdr{};
  hdr.max_drops = max_drops;
  hdr.nx = h->p.nx;
  hdr.ny = h->p.ny;
  hdr.periodic_y = h->p.periodic_y;
  hdr.ncx = L.ncx;
  hdr.ncy = L.ncy;
  // The launches from the rho_1 pass to the link list depend only on the lattice, the workspace, the
  // droplet bound, the threshold and the current buffer: they are captured once per such key into a
  // CUDA graph and replayed (four keys are kept, replaced in turn).
  lb_handle::DropGraph* dg = nullptr;
  for (auto& c : h->dgraph)
    if (c.exec && c.ws == d_ws && c.max_drops == max_drops && c.threshold == threshold && c.cur == h->cur) dg = &c;
  if (!dg) {
    dg = &h->dgraph[h->dgraph_next];
    h->dgraph_next = (h->dgraph_next + 1) % 4;
    if (dg->exec) cudaGraphExecDestroy(dg->exec);
    *dg = lb_handle::DropGraph{};
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = enqueue_analysis(h, v, L, hdr, threshold, max_drops, h->cap);
      e = cudaStreamEndCapture(h->cap, &graph);
      if (e1 != cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&dg->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      dg->exec = nullptr;
      return dfail(h, LB_ECUDA, "lb_droplets capture", e);
    }
    dg->ws = d_ws;
    dg->max_drops = max_drops;
    dg->threshold = threshold;
    dg->cur = h->cur;
  }
  const cudaError_t e = cudaGraphLaunch(dg->exec, h->stream);
  if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets", e);
  Header got{};
  if (int rc = read_header(h, v.hdr, &got)) return rc;
  if (got.err & kErrUnion) return dfail(h, LB_ECUDA, "droplet labelling did not converge");
  if (got.err & kErrDrops) return dfail(h, LB_ENOSPACE, "more droplets than max_drops");
  if (got.err & kErrDegree) return dfail(h, LB_ENOSPACE, "a droplet has more Voronoi neighbours than the adjacency holds");
  if (n_drops) *n_drops = got.n_drops;
  if (n_links) *n_links = got.n_links;
  return LB_OK;
}

int lb_droplets_get(lb_handle* h, const void* d_ws, size_t ws_bytes, double* cx, double* cy, long long* size,
                    int* links, int* label, int* color) {
  if (!h || !d_ws) return LB_EINVAL;
  Header hd{};
  if (int rc = read_header(h, d_ws, &hd)) return rc;
  DLayout L;
  if (hd.max_drops < 1 || hd.nx != h->p.nx || hd.ny != h->p.ny || !check_ws(h, d_ws, ws_bytes, hd.max_drops, &L))
    return dfail(h, LB_EINVAL, "workspace does not hold a droplet analysis of this lattice");
  const DView v = view(const_cast<void*>(d_ws), L);
  cudaStream_t s = h->stream;
  const size_t M = (size_t)hd.n_drops, N = (size_t)L.N;
  cudaError_t e = cudaSuccess;
  if (cx && M) e = cudaMemcpyAsync(cx, v.cx, M * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && cy && M) e = cudaMemcpyAsync(cy, v.cy, M * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && size && M) e = cudaMemcpyAsync(size, v.cnt, M * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && links && hd.n_links)
    e = cudaMemcpyAsync(links, v.links, (size_t)hd.n_links * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && label) e = cudaMemcpyAsync(label, v.did, N * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && color) e = cudaMemcpyAsync(color, v.col, N * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets_get", e);
  return LB_OK;
}

int lb_droplets_nusselt(lb_handle* h, const void* d_ws, size_t ws_bytes, double* nu) {
  if (!h || !d_ws || !nu) return LB_EINVAL;
  Header hd{};
  if (int rc = read_header(h, d_ws, &hd)) return rc;
  DLayout L;
  if (hd.max_drops < 1 || hd.nx != h->p.nx || hd.ny != h->p.ny || !check_ws(h, d_ws, ws_bytes, hd.max_drops, &L))
    return dfail(h, LB_EINVAL, "workspace does not hold a droplet analysis of this lattice");
  const int M = hd.n_drops;
  if (M == 0) return LB_OK;
  const double dT = h->p.T_down - h->p.T_up;
  if (h->p.periodic_y || dT == 0.0) {
    for (int i = 0; i < M; ++i) nu[i] = 0.0;
    return LB_OK;
  }
  const DView v = view(const_cast<void*>(d_ws), L);
  const Geo g{h->p.nx, h->p.ny, h->p.periodic_y, h->cfg.mask};
  double* stage = static_cast<double*>(h->buf[h->cur ^ 1]);
  double* dnu = stage + 5 * L.N;  // the staging buffer holds at least 9 doubles per node
  const double kappa = (h->p.tau_g - 0.5) / 3.0;
  const double den = kappa * (dT / (double)(h->p.ny - 2));
  cudaError_t e = fields_into(h, stage);
  if (e == cudaSuccess) {
    droplet_nusselt<<<nb(M, 256), 256, 0, h->stream>>>(g, M, v.cx, v.cy, stage, kappa, den, h->p.T_down, h->p.T_up, dnu);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(nu, dnu, (size_t)M * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets_nusselt", e);
  return LB_OK;
}

int lb_droplets_compare(lb_handle* h, const void* d_ws_prev, const void* d_ws_now, size_t ws_bytes, double d_max,
                        void* d_scratch, size_t scratch_bytes, int* counts4, int* broken, int* arising, int* t1,
                        int cap) {
  if (!h || !d_ws_prev || !d_ws_now || !counts4 || !d_scratch || cap < 0) return LB_EINVAL;
  Header hp{}, hn{};
  if (int rc = read_header(h, d_ws_prev, &hp)) return rc;
  if (int rc = read_header(h, d_ws_now, &hn)) return rc;
  DLayout Lp, Ln;
  if (hp.max_drops < 1 || hn.max_drops < 1 || hp.nx != h->p.nx || hn.nx != h->p.nx || hp.ny != h->p.ny ||
      hn.ny != h->p.ny || !check_ws(h, d_ws_prev, ws_bytes, hp.max_drops, &Lp) ||
      !check_ws(h, d_ws_now, ws_bytes, hn.max_drops, &Ln))
    return dfail(h, LB_EINVAL, "workspaces do not hold droplet analyses of this lattice");
  const int Mp = hp.n_drops, Mn = hn.n_drops;
  // scratch: near_np, n2p (per now droplet), near_pn, p2n (per prev droplet), count / offset / scan
  // blocks of the broken, arising and T1 lists, and the three lists
  const int Mx = Mp > Mn ? Mp : Mn;
  const size_t lmax = (size_t)Mx * kMaxDeg / 2 + 1;
  unsigned char* sp = static_cast<unsigned char*>(d_scratch);
  size_t used = 0;
  auto take = [&](size_t bytes) {
    int* p = reinterpret_cast<int*>(sp + used);
    used += round_up(bytes, kAlign);
    return p;
  };
  int* near_np = take((size_t)Mn * 4);
  int* n2p = take((size_t)Mn * 4);
  int* near_pn = take((size_t)Mp * 4);
  int* p2n = take((size_t)Mp * 4);
  int* cnt[3];
  int* off[3];
  int* blk[3];
  for (int k = 0; k < 3; ++k) {
    cnt[k] = take((lmax + 1) * 4);
    off[k] = take((lmax + 1) * 4);
    blk[k] = take((size_t)(nb((long long)lmax, kScanBlock) + 1) * 4);
  }
  int* dbroken = take(lmax * 8);
  int* darising = take(lmax * 8);
  int* dt1 = take(lmax * 16);
  if (scratch_bytes < used || ((uintptr_t)d_scratch % kAlign) != 0) {
    counts4[0] = (int)((used + 1023) / 1024);  // KiB needed
    return dfail(h, LB_ENOSPACE, "compare scratch too small or misaligned (counts4[0] = KiB needed)");
  }
  const DView vp = view(const_cast<void*>(d_ws_prev), Lp), vn = view(const_cast<void*>(d_ws_now), Ln);
  const Geo g{h->p.nx, h->p.ny, h->p.periodic_y, h->cfg.mask};
  const Grid Gp = grid_of(vp, Lp, h->p), Gn = grid_of(vn, Ln, h->p);
  cudaStream_t s = h->stream;
  const int T = 256;
  const double d2max = d_max * d_max;
  cudaError_t e = cudaMemsetAsync(p2n, 0xff, (size_t)Mp * 4, s);
  if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets_compare", e);
  if (Mn > 0) nearest_other<<<nb(Mn, T), T, 0, s>>>(g, Gp, Mn, vn.cx, vn.cy, d2max, near_np);
  if (Mp > 0) nearest_other<<<nb(Mp, T), T, 0, s>>>(g, Gn, Mp, vp.cx, vp.cy, d2max, near_pn);
  if (Mn > 0) {
    mutual<<<nb(Mn, T), T, 0, s>>>(Mn, near_np, near_pn, n2p);
    invert<<<nb(Mn, T), T, 0, s>>>(Mn, n2p, p2n);
  }
  // broken (per prev droplet) and arising (per now droplet): count, scan, write
  int tot[3] = {0, 0, 0};
  const int nsrc[2] = {Mp, Mn};
  for (int mode = 0; mode < 2; ++mode) {
    const int n = nsrc[mode];
    if (n == 0) continue;
    const DView& self = mode == 0 ? vp : vn;
    const DView& other = mode == 0 ? vn : vp;
    const int* map = mode == 0 ? p2n : n2p;
    int* outp = mode == 0 ? dbroken : darising;
    link_changes<<<nb(n, T), T, 0, s>>>(mode, n, self.adj, self.deg, other.adj, other.deg, map, nullptr, cnt[mode], nullptr);
    e = exclusive_scan(cnt[mode], n, off[mode], blk[mode], s);
    if (e == cudaSuccess) {
      link_changes<<<nb(n, T), T, 0, s>>>(mode, n, self.adj, self.deg, other.adj, other.deg, map, off[mode], nullptr, outp);
      e = cudaMemcpyAsync(&tot[mode], blk[mode] + nb(n, kScanBlock), sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets_compare", e);
  }
  if (tot[0] > 0) {
    t1_events<<<nb(tot[0], T), T, 0, s>>>(tot[0], dbroken, vp.adj, vp.deg, vn.adj, vn.deg, p2n, nullptr, cnt[2], nullptr,
                                          0);
    e = exclusive_scan(cnt[2], tot[0], off[2], blk[2], s);
    if (e == cudaSuccess) {
      t1_events<<<nb(tot[0], T), T, 0, s>>>(tot[0], dbroken, vp.adj, vp.deg, vn.adj, vn.deg, p2n, off[2], nullptr, dt1,
                                            (long long)lmax);
      e = cudaMemcpyAsync(&tot[2], blk[2] + nb(tot[0], kScanBlock), sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets_compare t1", e);
  }
  // matched count
  std::vector<int> n2p_h((size_t)Mn);
  if (Mn > 0) {
    e = cudaMemcpyAsync(n2p_h.data(), n2p, (size_t)Mn * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets_compare", e);
  }
  int matched = 0;
  for (int j = 0; j < Mn; ++j) matched += n2p_h[j] >= 0 ? 1 : 0;
  counts4[0] = matched;
  counts4[1] = tot[0];
  counts4[2] = tot[1];
  counts4[3] = tot[2];
  if (broken && tot[0]) e = cudaMemcpyAsync(broken, dbroken, (size_t)(tot[0] < cap ? tot[0] : cap) * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && arising && tot[1])
    e = cudaMemcpyAsync(arising, darising, (size_t)(tot[1] < cap ? tot[1] : cap) * 8, cudaMemcpyDeviceToHost, s);
  const int t1_held = tot[2] < (int)lmax ? tot[2] : (int)lmax;  // the device list keeps the first lmax events
  if (e == cudaSuccess && t1 && t1_held)
    e = cudaMemcpyAsync(t1, dt1, (size_t)(t1_held < cap ? t1_held : cap) * 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return dfail(h, LB_ECUDA, "lb_droplets_compare", e);
  return LB_OK;
}

}  // extern "C"
