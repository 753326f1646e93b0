// Grid construction: spherical (or box) Dirichlet domain, b^3 bricks, blockwise
// Hilbert space-filling-curve order of the bricks (SFC paragraph after Table I of
// arXiv 2303.00790; the curve construction is J. Skilling, "Programming the Hilbert
// curve", AIP Conf. Proc. 707, 381 (2004)).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "kscf_internal.h"

namespace kscf {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char* last_error() { return g_last_error.c_str(); }

// Hilbert index of a point of an n-dimensional 2^bits cube (Skilling 2004): the
// axes are converted in place to the "transposed" Hilbert index (inverse undo of the
// excess work, then Gray encoding), whose bits are then interleaved most
// significant first, axis 0 first.
static uint64_t hilbert_index3(uint32_t x0, uint32_t x1, uint32_t x2, int bits) {
  uint32_t X[3] = {x0, x1, x2};
  const int n = 3;
  if (bits <= 0) return 0;
  uint32_t M = 1u << (bits - 1);
  for (uint32_t Q = M; Q > 1; Q >>= 1) {
    uint32_t P = Q - 1;
    for (int i = 0; i < n; i++) {
      if (X[i] & Q) {
        X[0] ^= P;
      } else {
        uint32_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  for (int i = 1; i < n; i++) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (uint32_t Q = M; Q > 1; Q >>= 1)
    if (X[n - 1] & Q) t ^= Q - 1;
  for (int i = 0; i < n; i++) X[i] ^= t;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; b--)
    for (int i = 0; i < n; i++) h = (h << 1) | ((X[i] >> b) & 1u);
  return h;
}

uint64_t hilbert3_for_tests(uint32_t x, uint32_t y, uint32_t z, int bits) {
  return hilbert_index3(x, y, z, bits);
}

// in_domain(i,j,k) decides membership; lo/hi bound all member points.
template <typename F>
static int build(Grid& g, const int lo[3], const int hi[3], double h, const double center[3], int B,
                 F in_domain) {
  g.h = h;
  for (int a = 0; a < 3; a++) {
    g.center[a] = center[a];
    g.lo[a] = lo[a];
    g.ext[a] = hi[a] - lo[a] + 1;
    g.nb[a] = (g.ext[a] + B - 1) / B;
  }
  g.B = B;
  const int64_t nbox = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
  // count points per box brick and the lexicographic numbering
  std::vector<int64_t> count(nbox, 0);
  int64_t npts = 0;
  for (int k = lo[2]; k <= hi[2]; k++)
    for (int j = lo[1]; j <= hi[1]; j++)
      for (int i = lo[0]; i <= hi[0]; i++)
        if (in_domain(i, j, k)) {
          int64_t b = ((int64_t)((k - lo[2]) / B) * g.nb[1] + (j - lo[1]) / B) * g.nb[0] + (i - lo[0]) / B;
          count[b]++;
          npts++;
        }
  g.n_points = npts;
  // kept bricks ordered along the Hilbert curve
  int maxn = std::max(g.nb[0], std::max(g.nb[1], g.nb[2]));
  int bits = 0;
  while ((1 << bits) < maxn) bits++;
  std::vector<std::pair<uint64_t, int64_t>> keyed;
  for (int64_t b = 0; b < nbox; b++)
    if (count[b] > 0) {
      uint32_t bx = (uint32_t)(b % g.nb[0]);
      uint32_t by = (uint32_t)((b / g.nb[0]) % g.nb[1]);
      uint32_t bz = (uint32_t)(b / ((int64_t)g.nb[0] * g.nb[1]));
      keyed.push_back({hilbert_index3(bx, by, bz, bits), b});
    }
  std::sort(keyed.begin(), keyed.end());
  g.n_bricks = (int64_t)keyed.size();
  const int64_t b3 = (int64_t)B * B * B;
  g.n_slots = g.n_bricks * b3;
  g.brick_of_box.assign(nbox, -1);
  g.brick_xyz.resize(3 * g.n_bricks);
  for (int64_t r = 0; r < g.n_bricks; r++) {
    int64_t b = keyed[r].second;
    g.brick_of_box[b] = (int32_t)r;
    g.brick_xyz[3 * r + 0] = (int32_t)(b % g.nb[0]);
    g.brick_xyz[3 * r + 1] = (int32_t)((b / g.nb[0]) % g.nb[1]);
    g.brick_xyz[3 * r + 2] = (int32_t)(b / ((int64_t)g.nb[0] * g.nb[1]));
  }
  // face neighbours
  g.nbr.assign(6 * g.n_bricks, -1);
  for (int64_t r = 0; r < g.n_bricks; r++) {
    int bc[3] = {g.brick_xyz[3 * r], g.brick_xyz[3 * r + 1], g.brick_xyz[3 * r + 2]};
    for (int a = 0; a < 3; a++)
      for (int s = 0; s < 2; s++) {
        int c[3] = {bc[0], bc[1], bc[2]};
        c[a] += s ? 1 : -1;
        if (c[a] < 0 || c[a] >= g.nb[a]) continue;
        g.nbr[6 * r + 2 * a + s] = g.brick_of_box[((int64_t)c[2] * g.nb[1] + c[1]) * g.nb[0] + c[0]];
      }
  }
  // slot tables
  g.lex_of_slot.assign(g.n_slots, -1);
  g.mask.assign(g.n_slots, 0);
  int64_t lex = 0;
  for (int k = lo[2]; k <= hi[2]; k++)
    for (int j = lo[1]; j <= hi[1]; j++)
      for (int i = lo[0]; i <= hi[0]; i++)
        if (in_domain(i, j, k)) {
          int64_t s = g.slot_of(i, j, k);
          g.lex_of_slot[s] = lex++;
          g.mask[s] = 1;
        }
  return KSCF_OK;
}

}  // namespace kscf

using namespace kscf;

extern "C" const char* kscf_last_error(void) { return kscf::last_error(); }

extern "C" uint64_t kscf_launch_counter(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" int kscf_build_grid(const double center[3], double radius, double h, int brick,
                               kscf_grid** out) {
  if (!center || !out || !(radius > 0) || !(h > 0) || (brick != 8 && brick != 16)) {
    set_error("kscf_build_grid: invalid argument (radius>0, h>0, brick in {8,16}, non-null)");
    return KSCF_ERR_INVALID;
  }
  const double lim = radius * radius / (h * h) + 1e-9;
  const int n = (int)std::floor(radius / h) + 1;
  if (n > 4000) {
    set_error("kscf_build_grid: radius/h too large");
    return KSCF_ERR_INVALID;
  }
  // exact bounding box of the member points
  int nmax = 0;
  for (int i = 0; i <= n; i++)
    if ((double)((int64_t)i * i) <= lim) nmax = i;
  int lo[3] = {-nmax, -nmax, -nmax}, hi[3] = {nmax, nmax, nmax};
  kscf_grid* g = new (std::nothrow) kscf_grid();
  if (!g) {
    set_error("kscf_build_grid: host allocation failed");
    return KSCF_ERR_HOST_ALLOC;
  }
  try {
    build(g->g, lo, hi, h, center, brick, [lim](int i, int j, int k) {
      int64_t n2 = (int64_t)i * i + (int64_t)j * j + (int64_t)k * k;
      return (double)n2 <= lim;
    });
  } catch (const std::bad_alloc&) {
    delete g;
    set_error("kscf_build_grid: host allocation failed");
    return KSCF_ERR_HOST_ALLOC;
  }
  *out = g;
  return KSCF_OK;
}

extern "C" int kscf_build_grid_box(int nx, int ny, int nz, double h, int brick, kscf_grid** out) {
  if (!out || nx <= 0 || ny <= 0 || nz <= 0 || !(h > 0) || (brick != 8 && brick != 16) ||
      nx > 8192 || ny > 8192 || nz > 8192) {
    set_error("kscf_build_grid_box: invalid argument");
    return KSCF_ERR_INVALID;
  }
  int lo[3] = {0, 0, 0}, hi[3] = {nx - 1, ny - 1, nz - 1};
  double c[3] = {0, 0, 0};
  kscf_grid* g = new (std::nothrow) kscf_grid();
  if (!g) {
    set_error("kscf_build_grid_box: host allocation failed");
    return KSCF_ERR_HOST_ALLOC;
  }
  try {
    build(g->g, lo, hi, h, c, brick, [](int, int, int) { return true; });
  } catch (const std::bad_alloc&) {
    delete g;
    set_error("kscf_build_grid_box: host allocation failed");
    return KSCF_ERR_HOST_ALLOC;
  }
  *out = g;
  return KSCF_OK;
}

static void fill_info(const Grid& g, kscf_grid_info* info) {
  std::memset(info, 0, sizeof(*info));
  info->n_points = g.n_points;
  info->n_slots = g.n_slots;
  info->n_bricks = g.n_bricks;
  info->brick = g.B;
  for (int a = 0; a < 3; a++) {
    info->lo[a] = g.lo[a];
    info->extent[a] = g.ext[a];
    info->center[a] = g.center[a];
  }
  info->h = g.h;
}

namespace kscf {
void grid_info(const Grid& g, kscf_grid_info* info) { fill_info(g, info); }
}

extern "C" int kscf_grid_get_info(const kscf_grid* grid, kscf_grid_info* info) {
  if (!grid || !info) {
    set_error("kscf_grid_get_info: null argument");
    return KSCF_ERR_INVALID;
  }
  fill_info(grid->g, info);
  return KSCF_OK;
}

extern "C" int kscf_grid_slots(const kscf_grid* grid, int64_t* lex_of_slot, int32_t* ijk_of_slot) {
  if (!grid) {
    set_error("kscf_grid_slots: null grid");
    return KSCF_ERR_INVALID;
  }
  const Grid& g = grid->g;
  if (lex_of_slot) std::memcpy(lex_of_slot, g.lex_of_slot.data(), sizeof(int64_t) * g.n_slots);
  if (ijk_of_slot)
    for (int64_t s = 0; s < g.n_slots; s++) g.slot_ijk(s, ijk_of_slot + 3 * s);
  return KSCF_OK;
}

extern "C" int kscf_grid_free(kscf_grid* grid) {
  delete grid;
  return KSCF_OK;
}

// Hilbert index of brick coordinates, exported for the host-logic tests.
extern "C" uint64_t kscf_hilbert_index3(uint32_t x, uint32_t y, uint32_t z, int bits) {
  return kscf::hilbert3_for_tests(x, y, z, bits);
}
