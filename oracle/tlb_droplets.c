/*
 * Plain CPU oracle of the droplet-topology analysis of TLBfind (arXiv 2109.12565, Sec. 2.4
 * "Delaunay triangulation"): droplet regions, their centres of mass, the digital Voronoi
 * tessellation coloured by the nearest centre, and the Delaunay links read off the points where
 * digital Voronoi cells meet.
 *
 * TEST INFRASTRUCTURE ONLY (see tlb_oracle.c).  Written to be checked by eye against the
 * definitions below, not for speed: labelling is a breadth-first flood fill, the Voronoi colouring
 * compares every node with every centre.
 *
 * Definitions (readings of Sec. 2.4; the paper names the steps but not these details):
 *   D1  a droplet node is a fluid node with rho_1 > B_th (strict);
 *   D2  droplet nodes are connected through the 4 nearest neighbours, x periodic, y periodic when
 *       periodic_y;
 *   D3  droplets are numbered 0, 1, ... in the order of their smallest node index y * nx + x;
 *   D4  the centre of a droplet is the plain mean of its node coordinates, each unwrapped
 *       relative to the droplet's smallest node (x offsets in (-nx/2, nx/2], likewise y when
 *       periodic), then wrapped into [0, nx) (and [0, ny));
 *   D5  every fluid node takes the id of the nearest centre: distance^2 = dx * dx + dy * dy in
 *       double precision, dx = x - c_x taken to its periodic image in [-nx/2, nx/2], ties to the
 *       smaller id; solid nodes take -1;
 *   D6  links: in every 2 x 2 window of fluid nodes (x, y), (x+1, y), (x, y+1), (x+1, y+1) (x + 1
 *       periodic, y + 1 periodic or inside the lattice), three distinct colours give the three
 *       pairs, four distinct colours give the four pairs of neighbouring corners (the sides of the
 *       quadrilateral, not its diagonals).
 */
#include <stdlib.h>
#include <string.h>

#include "tlb_oracle.h"

static int wrapi(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

int orc_droplet_labels(const orc_params* prm, const uint8_t* mask, const double* rho1, double threshold, int* label,
                       int* n_drops) {
  if (!prm || prm->nx < 1 || prm->ny < 1 || !rho1 || !label || !n_drops) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  uint8_t* solid = malloc((size_t)N);
  int* queue = malloc((size_t)N * sizeof(int));
  if (!solid || !queue) {
    free(solid);
    free(queue);
    return -2;
  }
  orc_solid_map(prm, mask, solid);
  for (long n = 0; n < N; ++n) label[n] = -1;
  int next = 0;
  for (long n = 0; n < N; ++n) {
    if (solid[n] || !(rho1[n] > threshold) || label[n] >= 0) continue;
    /* n is the smallest node of a new droplet (D3): flood fill its component (D2) */
    long head = 0, tail = 0;
    label[n] = next;
    queue[tail++] = (int)n;
    while (head < tail) {
      const int m = queue[head++];
      const int x = m % nx, y = m / nx;
      const int nb[4][2] = {{x + 1, y}, {x - 1, y}, {x, y + 1}, {x, y - 1}};
      for (int k = 0; k < 4; ++k) {
        int xx = wrapi(nb[k][0], nx), yy = nb[k][1];
        if (prm->periodic_y) yy = wrapi(yy, ny);
        else if (yy < 0 || yy >= ny) continue;
        const long q = (long)yy * nx + xx;
        if (solid[q] || !(rho1[q] > threshold) || label[q] >= 0) continue;
        label[q] = next;
        queue[tail++] = (int)q;
      }
    }
    ++next;
  }
  *n_drops = next;
  free(solid);
  free(queue);
  return 0;
}

/* Offset a - b taken into (-n/2, n/2] (integer form of the minimum image). */
static long min_image_i(long d, int n) {
  if (2 * d > n) d -= n;
  if (2 * d <= -n) d += n;
  return d;
}

int orc_droplet_centres(const orc_params* prm, const int* label, int n_drops, double* cx, double* cy,
                        long long* size) {
  if (!prm || !label || n_drops < 0 || (n_drops > 0 && (!cx || !cy))) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  long* root = malloc((size_t)(n_drops > 0 ? n_drops : 1) * sizeof(long));
  long long* sx = calloc((size_t)(n_drops > 0 ? n_drops : 1), sizeof(long long));
  long long* sy = calloc((size_t)(n_drops > 0 ? n_drops : 1), sizeof(long long));
  long long* cnt = calloc((size_t)(n_drops > 0 ? n_drops : 1), sizeof(long long));
  if (!root || !sx || !sy || !cnt) {
    free(root), free(sx), free(sy), free(cnt);
    return -2;
  }
  for (int d = 0; d < n_drops; ++d) root[d] = -1;
  for (long n = 0; n < N; ++n) {
    const int d = label[n];
    if (d < 0) continue;
    if (d >= n_drops) {
      free(root), free(sx), free(sy), free(cnt);
      return -1;
    }
    if (root[d] < 0) root[d] = n; /* labels are met in increasing node order: the first is the smallest */
    const long rx = root[d] % nx, ry = root[d] / nx, x = n % nx, y = n / nx;
    sx[d] += min_image_i(x - rx, nx);
    sy[d] += prm->periodic_y ? min_image_i(y - ry, ny) : (y - ry);
    cnt[d] += 1;
  }
  for (int d = 0; d < n_drops; ++d) {
    const double rx = (double)(root[d] % nx), ry = (double)(root[d] / nx);
    double x = rx + (double)sx[d] / (double)cnt[d];
    double y = ry + (double)sy[d] / (double)cnt[d];
    if (x < 0.0) x += nx;
    else if (x >= nx) x -= nx;
    if (prm->periodic_y) {
      if (y < 0.0) y += ny;
      else if (y >= ny) y -= ny;
    }
    cx[d] = x;
    cy[d] = y;
    if (size) size[d] = cnt[d];
  }
  free(root), free(sx), free(sy), free(cnt);
  return 0;
}

int orc_digital_voronoi(const orc_params* prm, const uint8_t* mask, const double* cx, const double* cy, int n_drops,
                        int* color) {
  if (!prm || prm->nx < 1 || prm->ny < 1 || !color || n_drops < 0 || (n_drops > 0 && (!cx || !cy))) return -1;
  const int nx = prm->nx, ny = prm->ny;
  const long N = (long)nx * ny;
  uint8_t* solid = malloc((size_t)N);
  if (!solid) return -2;
  orc_solid_map(prm, mask, solid);
  const double hx = 0.5 * nx, hy = 0.5 * ny;
  for (long n = 0; n < N; ++n) {
    color[n] = -1;
    if (solid[n] || n_drops == 0) continue;
    const double x = (double)(n % nx), y = (double)(n / nx);
    double best = 0.0;
    int best_id = -1;
    for (int d = 0; d < n_drops; ++d) {
      double dx = x - cx[d];
      if (dx > hx) dx -= nx;
      else if (dx < -hx) dx += nx;
      double dy = y - cy[d];
      if (prm->periodic_y) {
        if (dy > hy) dy -= ny;
        else if (dy < -hy) dy += ny;
      }
      const double d2 = dx * dx + dy * dy;
      if (best_id < 0 || d2 < best) { /* ids ascend: a tie keeps the smaller id */
        best = d2;
        best_id = d;
      }
    }
    color[n] = best_id;
  }
  free(solid);
  return 0;
}

static int cmp_pair(const void* a, const void* b) {
  const int* p = a;
  const int* q = b;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}

int orc_voronoi_links(const orc_params* prm, const int* color, int* links, long max_links, long* n_links) {
  if (!prm || prm->nx < 1 || prm->ny < 1 || !color || !n_links || max_links < 0) return -1;
  const int nx = prm->nx, ny = prm->ny;
  long cap = 1024, n = 0;
  int* all = malloc((size_t)cap * 2 * sizeof(int));
  if (!all) return -2;
  const int ymax = prm->periodic_y ? ny : ny - 1;
  for (int y = 0; y < ymax; ++y)
    for (int x = 0; x < nx; ++x) {
      const int x1 = (x + 1) % nx, y1 = (y + 1) % ny;
      /* corners in cyclic order around the window: 00, 10, 11, 01 */
      const int c[4] = {color[(long)y * nx + x], color[(long)y * nx + x1], color[(long)y1 * nx + x1],
                        color[(long)y1 * nx + x]};
      if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[3] < 0) continue;
      int distinct[4], k = 0;
      for (int i = 0; i < 4; ++i) {
        int seen = 0;
        for (int j = 0; j < k; ++j) seen |= distinct[j] == c[i];
        if (!seen) distinct[k++] = c[i];
      }
      int pairs[4][2], np = 0;
      if (k == 3) {
        pairs[0][0] = distinct[0], pairs[0][1] = distinct[1];
        pairs[1][0] = distinct[1], pairs[1][1] = distinct[2];
        pairs[2][0] = distinct[0], pairs[2][1] = distinct[2];
        np = 3;
      } else if (k == 4) {
        for (int i = 0; i < 4; ++i) pairs[i][0] = c[i], pairs[i][1] = c[(i + 1) % 4];
        np = 4;
      }
      for (int i = 0; i < np; ++i) {
        if (n == cap) {
          cap *= 2;
          int* g = realloc(all, (size_t)cap * 2 * sizeof(int));
          if (!g) {
            free(all);
            return -2;
          }
          all = g;
        }
        const int a = pairs[i][0], b = pairs[i][1];
        all[2 * n] = a < b ? a : b;
        all[2 * n + 1] = a < b ? b : a;
        ++n;
      }
    }
  qsort(all, (size_t)n, 2 * sizeof(int), cmp_pair);
  long u = 0;
  for (long i = 0; i < n; ++i) {
    if (u > 0 && all[2 * (u - 1)] == all[2 * i] && all[2 * (u - 1) + 1] == all[2 * i + 1]) continue;
    all[2 * u] = all[2 * i];
    all[2 * u + 1] = all[2 * i + 1];
    ++u;
  }
  *n_links = u;
  if (links)
    for (long i = 0; i < u && i < max_links; ++i) {
      links[2 * i] = all[2 * i];
      links[2 * i + 1] = all[2 * i + 1];
    }
  free(all);
  return u > max_links && links ? -3 : 0;
}
