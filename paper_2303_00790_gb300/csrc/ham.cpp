// Hamiltonian tables: order-12 finite-difference weights, synthetic local potential
// and Kleinman-Bylander projector tables in slot (Hilbert-brick) order.
// (arXiv 2303.00790: Intro -- high-order finite differences in real space;
//  Computational details -- norm-conserving pseudopotentials in KB form.)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "kscf_internal.h"

namespace kscf {
void grid_info(const Grid& g, kscf_grid_info* info);
}

using namespace kscf;

// Central weights of the order-12 second derivative,
//   f''(0) ~ h^-2 [w0 f(0) + sum_{k=1..6} w_k (f(kh) + f(-kh))],
// w_k = 2 (-1)^(k+1) (6!)^2 / (k^2 (6-k)! (6+k)!), w0 = -2 sum_k w_k.
static const double kW12[7] = {-5369.0 / 1800.0, 12.0 / 7.0,  -15.0 / 56.0,   10.0 / 189.0,
                               -1.0 / 112.0,     2.0 / 1925.0, -1.0 / 16632.0};

template <typename T>
static cudaError_t upload(T** dst, const T* src, size_t n) {
  *dst = nullptr;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
}

static void free_ham(Ham& H) {
  void* ptrs[] = {H.d_nbr,           H.d_mask,         H.d_lex,          H.d_pad,          H.d_live,
                  H.d_vion,          H.d_v64,           H.d_v32,          H.d_kb_atom_ptr,  H.d_kb_atom_slot,
                  H.d_kb_atom_chi64, H.d_kb_atom_chi32, H.d_kb_slot_ptr, H.d_kb_slot_atom,
                  H.d_kb_slot_chi64, H.d_kb_slot_chi32, H.d_kb_energy, H.d_kb_entry_lslot,
                  H.d_lines,         H.d_nlines,        H.d_brick_atoms, H.d_brick_natoms, H.d_kb_entry_word};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (H.cell_tables_own) {
    void* cell[] = {H.d_cell_nbr, H.d_cell_kb_ptr, H.d_cell_kb_chi32, H.d_cell_kb_atom};
    for (void* p : cell)
      if (p) cudaFree(p);
  }
}

extern "C" int kscf_ham_free(kscf_ham* ham) {
  if (!ham) return KSCF_OK;
  free_ham(ham->h);
  delete ham;
  return KSCF_OK;
}

namespace {
struct KBEntry {
  int64_t slot;
  int32_t atom;
  double chi[4];
};

// slot of the cell-local point r = x + 8 y + 64 z of cell c (bricks of B = 8 or 16 points;
// a 16^3 brick holds the cells brick * 8 + ox + 2 oy + 4 oz, points x-fastest in the brick)
int64_t cell_slot(int B, int64_t c, int r) {
  if (B == 8) return c * 512 + r;
  const int o = (int)(c & 7);
  const int x = (o & 1) * 8 + (r & 7), y = ((o >> 1) & 1) * 8 + ((r >> 3) & 7), z = (o >> 2) * 8 + (r >> 6);
  return (c >> 3) * 4096 + ((int64_t)z * 16 + y) * 16 + x;
}
}  // namespace

extern "C" int kscf_build_hamiltonian(const kscf_grid* grid, const kscf_atom* atoms, int n_atoms,
                                      const kscf_species* species, int n_species, kscf_ham** out) {
  if (!grid || !out || n_atoms < 0 || (n_atoms > 0 && !atoms) || n_species < 0 ||
      (n_species > 0 && !species)) {
    set_error("kscf_build_hamiltonian: invalid argument");
    return KSCF_ERR_INVALID;
  }
  // species lookup and validation
  std::vector<int> sp_of_atom(n_atoms);
  for (int a = 0; a < n_atoms; a++) {
    int found = -1;
    for (int s = 0; s < n_species; s++)
      if (species[s].z_number == atoms[a].z_number) found = s;
    if (found < 0) {
      set_error("kscf_build_hamiltonian: no species for atom %d (Z=%d)", a, atoms[a].z_number);
      return KSCF_ERR_INVALID;
    }
    const kscf_species& s = species[found];
    if ((s.n_proj != 0 && s.n_proj != 4) || !(s.r_c > 0) || !(s.r_gauss > 0) ||
        (s.n_proj == 4 && (!(s.r_p > 0) || !(s.r_cut > 0)))) {
      set_error("kscf_build_hamiltonian: invalid species parameters (Z=%d)", s.z_number);
      return KSCF_ERR_INVALID;
    }
    sp_of_atom[a] = found;
  }
  kscf_ham* hh = new (std::nothrow) kscf_ham();
  if (!hh) {
    set_error("kscf_build_hamiltonian: host allocation failed");
    return KSCF_ERR_HOST_ALLOC;
  }
  Ham& H = hh->h;
  int rc = KSCF_OK;
  try {
    H.grid = grid->g;
    const Grid& g = H.grid;
    const double h = g.h;
    for (int k = 0; k <= 6; k++) H.stencil[k] = -0.5 * kW12[k] / (h * h);
    cudaGetDevice(&H.device);

    // ---- geometry tables ----
    std::vector<int64_t> pad;
    std::vector<int32_t> live;
    for (int64_t s = 0; s < g.n_slots; s++) {
      if (!g.mask[s]) pad.push_back(s);
      else live.push_back((int32_t)s);
    }
    H.n_pad = (int64_t)pad.size();
    H.n_live = (int64_t)live.size();
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = upload(&H.d_nbr, g.nbr.data(), g.nbr.size());
    if (e == cudaSuccess) e = upload(&H.d_mask, g.mask.data(), g.mask.size());
    if (e == cudaSuccess) e = upload(&H.d_lex, g.lex_of_slot.data(), g.lex_of_slot.size());
    if (e == cudaSuccess) e = upload(&H.d_pad, pad.data(), pad.size());
    if (e == cudaSuccess) e = upload(&H.d_live, live.data(), live.size());
    if ((g.B == 8 || g.B == 16) && e == cudaSuccess) {
      // cells of the chunk-major filter: neighbours across the six faces (inside a 16^3
      // brick the adjacent octant, else the octant of the neighbour brick that touches it)
      const int per = g.B == 8 ? 1 : 8;
      H.n_cells = g.n_bricks * per;
      std::vector<int32_t> cnbr((size_t)H.n_cells * 6, -1);
      for (int64_t c = 0; c < H.n_cells; c++) {
        const int64_t b = c / per;
        const int o = (int)(c % per);
        for (int f = 0; f < 6; f++) {
          if (per == 1) {
            cnbr[c * 6 + f] = g.nbr[b * 6 + f];
            continue;
          }
          const int ax = f >> 1, up = f & 1, oa = (o >> ax) & 1;
          const int o2 = o ^ (1 << ax);
          if (oa != up) {
            cnbr[c * 6 + f] = (int32_t)(b * 8 + o2);
          } else {
            const int32_t nb = g.nbr[b * 6 + f];
            cnbr[c * 6 + f] = nb < 0 ? -1 : (int32_t)((int64_t)nb * 8 + o2);
          }
        }
      }
      // live lines per cell and pass: x lines (y, z), y lines (x, z), z lines (x, y)
      std::vector<uint8_t> lines((size_t)H.n_cells * 3 * 64, 0), nlines((size_t)H.n_cells * 3, 0);
      for (int64_t c = 0; c < H.n_cells; c++) {
        for (int pass = 0; pass < 3; pass++) {
          int n = 0;
          for (int bb = 0; bb < 8; bb++)
            for (int aa = 0; aa < 8; aa++) {
              bool live = false;
              for (int t = 0; t < 8; t++) {
                int x, y, z;
                if (pass == 0) { x = t; y = aa; z = bb; }
                else if (pass == 1) { x = aa; y = t; z = bb; }
                else { x = aa; y = bb; z = t; }
                live |= g.mask[cell_slot(g.B, c, (z * 8 + y) * 8 + x)] != 0;
              }
              if (live) lines[(c * 3 + pass) * 64 + n++] = (uint8_t)(aa + 8 * bb);
            }
          nlines[c * 3 + pass] = (uint8_t)n;
        }
      }
      e = upload(&H.d_lines, lines.data(), lines.size());
      if (e == cudaSuccess) e = upload(&H.d_nlines, nlines.data(), nlines.size());
      if (per == 1) {
        H.d_cell_nbr = H.d_nbr;
      } else {
        H.cell_tables_own = true;
        if (e == cudaSuccess) e = upload(&H.d_cell_nbr, cnbr.data(), cnbr.size());
      }
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&H.d_v64, sizeof(double) * g.n_slots);
    if (e == cudaSuccess) e = cudaMalloc((void**)&H.d_v32, sizeof(float) * g.n_slots);
    if (e != cudaSuccess) {
      set_error("kscf_build_hamiltonian: device upload failed: %s", cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
      throw 1;
    }

    // ---- local potential on the device ----
    std::vector<double> at(8 * (size_t)std::max(n_atoms, 1));
    for (int a = 0; a < n_atoms; a++) {
      const kscf_species& s = species[sp_of_atom[a]];
      double* r = &at[8 * a];
      r[0] = atoms[a].x; r[1] = atoms[a].y; r[2] = atoms[a].z;
      r[3] = s.z_valence; r[4] = s.r_c; r[5] = s.a_gauss; r[6] = s.r_gauss; r[7] = 0.0;
    }
    std::vector<double> xyz(3 * (size_t)g.n_slots);
    for (int64_t sl = 0; sl < g.n_slots; sl++) {
      int ijk[3];
      g.slot_ijk(sl, ijk);
      for (int d = 0; d < 3; d++) xyz[3 * sl + d] = g.center[d] + h * (double)ijk[d];
    }
    double* d_at = nullptr;
    double* d_xyz = nullptr;
    e = upload(&d_at, at.data(), 8 * (size_t)n_atoms);
    if (e == cudaSuccess) e = upload(&d_xyz, xyz.data(), xyz.size());
    if (e == cudaSuccess) e = launch_vloc(H, d_xyz, d_at, n_atoms, 0);
    if (e == cudaSuccess) e = launch_v_to_f32(H, 0);
    if (e == cudaSuccess) e = cudaMalloc((void**)&H.d_vion, sizeof(double) * g.n_slots);
    if (e == cudaSuccess) e = cudaMemcpyAsync(H.d_vion, H.d_v64, sizeof(double) * g.n_slots, cudaMemcpyDeviceToDevice, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (d_at) cudaFree(d_at);
    if (d_xyz) cudaFree(d_xyz);
    if (e != cudaSuccess) {
      set_error("kscf_build_hamiltonian: local potential failed: %s", cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
      throw 1;
    }

    // ---- KB projector tables (host) ----
    std::vector<KBEntry> ent;
    std::vector<int64_t> atom_ptr(1, 0);
    std::vector<double> energy;
    int nkb = 0;
    for (int a = 0; a < n_atoms; a++) {
      const kscf_species& s = species[sp_of_atom[a]];
      if (s.n_proj == 0) continue;
      const double ax = atoms[a].x, ay = atoms[a].y, az = atoms[a].z;
      const double rcut = s.r_cut, rp = s.r_p;
      int lo[3], hi[3];
      const double pa[3] = {ax, ay, az};
      for (int d = 0; d < 3; d++) {
        lo[d] = (int)std::floor((pa[d] - g.center[d] - rcut) / h) - 1;
        hi[d] = (int)std::ceil((pa[d] - g.center[d] + rcut) / h) + 1;
      }
      size_t first = ent.size();
      for (int k = lo[2]; k <= hi[2]; k++)
        for (int j = lo[1]; j <= hi[1]; j++)
          for (int i = lo[0]; i <= hi[0]; i++) {
            int64_t sl = g.slot_of(i, j, k);
            if (sl < 0 || !g.mask[sl]) continue;
            const double x = g.center[0] + h * (double)i;
            const double y = g.center[1] + h * (double)j;
            const double z = g.center[2] + h * (double)k;
            const double dx = x - ax, dy = y - ay, dz = z - az;
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 <= rcut * rcut)) continue;
            const double gv = std::exp(-r2 / (2.0 * rp * rp));
            KBEntry en;
            en.slot = sl;
            en.atom = nkb;
            en.chi[0] = gv;
            en.chi[1] = dx / rp * gv;
            en.chi[2] = dy / rp * gv;
            en.chi[3] = dz / rp * gv;
            ent.push_back(en);
          }
      std::sort(ent.begin() + first, ent.end(),
                [](const KBEntry& p, const KBEntry& q) { return p.slot < q.slot; });
      atom_ptr.push_back((int64_t)ent.size());
      const double h3 = h * h * h;
      energy.push_back(s.e_s * h3);
      energy.push_back(s.e_p * h3);
      energy.push_back(s.e_p * h3);
      energy.push_back(s.e_p * h3);
      nkb++;
    }
    H.n_kb = nkb;
    H.n_kb_entries = (int64_t)ent.size();
    const int64_t ne = H.n_kb_entries;
    // per-atom arrays
    std::vector<int64_t> a_slot(ne);
    std::vector<double> a_chi(4 * ne);
    std::vector<float> a_chi32(4 * ne);
    for (int64_t q = 0; q < ne; q++) {
      a_slot[q] = ent[q].slot;
      for (int l = 0; l < 4; l++) {
        a_chi[4 * q + l] = ent[q].chi[l];
        a_chi32[4 * q + l] = (float)ent[q].chi[l];
      }
    }
    // per-slot CSR (counting sort by slot, stable in atom order)
    std::vector<int64_t> s_ptr(g.n_slots + 1, 0);
    for (int64_t q = 0; q < ne; q++) s_ptr[ent[q].slot + 1]++;
    for (int64_t s = 0; s < g.n_slots; s++) s_ptr[s + 1] += s_ptr[s];
    std::vector<int64_t> fill(s_ptr.begin(), s_ptr.end() - 1);
    std::vector<int32_t> s_atom(ne);
    std::vector<double> s_chi(4 * ne);
    std::vector<float> s_chi32(4 * ne);
    int maxe = 0;
    for (int64_t q = 0; q < ne; q++) {
      int64_t p = fill[ent[q].slot]++;
      s_atom[p] = ent[q].atom;
      for (int l = 0; l < 4; l++) {
        s_chi[4 * p + l] = ent[q].chi[l];
        s_chi32[4 * p + l] = (float)ent[q].chi[l];
      }
    }
    for (int64_t s = 0; s < g.n_slots; s++) maxe = std::max(maxe, (int)(s_ptr[s + 1] - s_ptr[s]));
    H.max_slot_entries = maxe;

    // Gershgorin bounds of V_NL through the projector Gram G_ij = h^3 <chi_i, chi_j>:
    // overlapping atom pairs (centre distance <= sum of cutoffs) are merged along
    // their slot-sorted entry lists.
    {
      const double h3 = h * h * h;
      std::vector<int> kb_atom(nkb);
      {
        int q = 0;
        for (int a = 0; a < n_atoms; a++)
          if (species[sp_of_atom[a]].n_proj != 0) kb_atom[q++] = a;
      }
      std::vector<double> row_pos(4 * (size_t)nkb, 0.0), row_neg(4 * (size_t)nkb, 0.0);
      for (int i1 = 0; i1 < nkb; i1++)
        for (int i2 = i1; i2 < nkb; i2++) {
          const kscf_atom &A1 = atoms[kb_atom[i1]], &A2 = atoms[kb_atom[i2]];
          const double reach = species[sp_of_atom[kb_atom[i1]]].r_cut + species[sp_of_atom[kb_atom[i2]]].r_cut;
          const double ddx = A1.x - A2.x, ddy = A1.y - A2.y, ddz = A1.z - A2.z;
          if (ddx * ddx + ddy * ddy + ddz * ddz > reach * reach * (1.0 + 1e-12)) continue;
          double blk[16] = {0};
          int64_t p = atom_ptr[i1], q = atom_ptr[i2];
          while (p < atom_ptr[i1 + 1] && q < atom_ptr[i2 + 1]) {
            if (ent[p].slot < ent[q].slot) { p++; continue; }
            if (ent[q].slot < ent[p].slot) { q++; continue; }
            for (int l1 = 0; l1 < 4; l1++)
              for (int l2 = 0; l2 < 4; l2++) blk[4 * l1 + l2] += ent[p].chi[l1] * ent[q].chi[l2];
            p++;
            q++;
          }
          for (int l1 = 0; l1 < 4; l1++)
            for (int l2 = 0; l2 < 4; l2++) {
              const double G = std::fabs(h3 * blk[4 * l1 + l2]);
              const double e1 = energy[4 * i1 + l1] / h3, e2 = energy[4 * i2 + l2] / h3;
              const double gp = std::sqrt(std::max(e1, 0.0) * std::max(e2, 0.0)) * G;
              const double gn = std::sqrt(std::max(-e1, 0.0) * std::max(-e2, 0.0)) * G;
              row_pos[4 * i1 + l1] += gp;
              row_neg[4 * i1 + l1] += gn;
              if (i2 != i1) {
                row_pos[4 * i2 + l2] += gp;
                row_neg[4 * i2 + l2] += gn;
              }
            }
        }
      H.kb_upper = 0.0;
      H.kb_lower = 0.0;
      for (size_t i = 0; i < row_pos.size(); i++) {
        H.kb_upper = std::max(H.kb_upper, row_pos[i]);
        H.kb_lower = std::max(H.kb_lower, row_neg[i]);
      }
    }

    e = cudaSuccess;
    if (e == cudaSuccess) e = upload(&H.d_kb_atom_ptr, atom_ptr.data(), atom_ptr.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_atom_slot, a_slot.data(), a_slot.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_atom_chi64, a_chi.data(), a_chi.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_atom_chi32, a_chi32.data(), a_chi32.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_slot_ptr, s_ptr.data(), s_ptr.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_slot_atom, s_atom.data(), s_atom.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_slot_chi64, s_chi.data(), s_chi.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_slot_chi32, s_chi32.data(), s_chi32.size());
    if (e == cudaSuccess) e = upload(&H.d_kb_energy, energy.data(), energy.size());
    {
      // entry (slot order) -> slot index inside its brick
      const int64_t b3 = (int64_t)g.B * g.B * g.B;
      std::vector<uint16_t> lslot(ne);
      for (int64_t s2 = 0; s2 < g.n_slots; s2++)
        for (int64_t q = s_ptr[s2]; q < s_ptr[s2 + 1]; q++) lslot[q] = (uint16_t)(s2 % b3);
      if (e == cudaSuccess) e = upload(&H.d_kb_entry_lslot, lslot.data(), lslot.size());
      if (H.n_cells > 0 && e == cudaSuccess) {
        // the entries in cell order (the slot order itself for 8^3 bricks), per-cell atom
        // lists and packed entry words for the chunk-major filter kernels
        const bool own = g.B != 8;
        std::vector<int64_t> cptr;
        std::vector<float> cchi;
        std::vector<int32_t> catom;
        std::vector<uint16_t> clocal(ne);
        if (own) {
          cptr.assign((size_t)H.n_cells * 512 + 1, 0);
          cchi.resize(4 * (size_t)ne);
          catom.resize(ne);
        }
        int64_t q2 = 0;
        for (int64_t c = 0; c < H.n_cells; c++)
          for (int r = 0; r < 512; r++) {
            const int64_t s2 = cell_slot(g.B, c, r);
            if (own) cptr[c * 512 + r] = q2;
            for (int64_t q = s_ptr[s2]; q < s_ptr[s2 + 1]; q++, q2++) {
              clocal[q2] = (uint16_t)r;
              if (own) {
                catom[q2] = s_atom[q];
                for (int l = 0; l < 4; l++) cchi[4 * q2 + l] = s_chi32[4 * q + l];
              }
            }
          }
        if (own) cptr[(size_t)H.n_cells * 512] = q2;
        const std::vector<int64_t>& cp = own ? cptr : s_ptr;
        const std::vector<int32_t>& ca = own ? catom : s_atom;
        const int64_t nc = H.n_cells;
        std::vector<int32_t> batoms((size_t)nc * KSCF_BRICK_ATOMS, -1), bnat(nc, 0);
        std::vector<uint32_t> word(ne);
        bool ok = true;
        for (int64_t c = 0; c < nc; c++) {
          for (int64_t q = cp[c * 512]; q < cp[(c + 1) * 512]; q++) {
            const int32_t at = ca[q];
            int li = 0;
            while (li < bnat[c] && batoms[c * KSCF_BRICK_ATOMS + li] != at) li++;
            if (li == bnat[c]) {
              if (bnat[c] == KSCF_BRICK_ATOMS) {
                ok = false;
                li = 0;
              } else {
                batoms[c * KSCF_BRICK_ATOMS + li] = at;
                bnat[c]++;
              }
            }
            word[q] = (uint32_t)clocal[q] | ((uint32_t)li << 16);
          }
        }
        H.brick_atoms_ok = ok;
        if (e == cudaSuccess) e = upload(&H.d_brick_atoms, batoms.data(), batoms.size());
        if (e == cudaSuccess) e = upload(&H.d_brick_natoms, bnat.data(), bnat.size());
        if (e == cudaSuccess) e = upload(&H.d_kb_entry_word, word.data(), word.size());
        if (own) {
          if (e == cudaSuccess) e = upload(&H.d_cell_kb_ptr, cptr.data(), cptr.size());
          if (e == cudaSuccess) e = upload(&H.d_cell_kb_chi32, cchi.data(), cchi.size());
          if (e == cudaSuccess) e = upload(&H.d_cell_kb_atom, catom.data(), catom.size());
        } else {
          H.d_cell_kb_ptr = H.d_kb_slot_ptr;
          H.d_cell_kb_chi32 = H.d_kb_slot_chi32;
          H.d_cell_kb_atom = H.d_kb_slot_atom;
        }
      }
    }
    if (e != cudaSuccess) {
      set_error("kscf_build_hamiltonian: KB upload failed: %s", cudaGetErrorString(e));
      rc = KSCF_ERR_CUDA;
      throw 1;
    }
  } catch (const std::bad_alloc&) {
    set_error("kscf_build_hamiltonian: host allocation failed");
    rc = KSCF_ERR_HOST_ALLOC;
  } catch (int) {
  }
  if (rc != KSCF_OK) {
    free_ham(H);
    delete hh;
    return rc;
  }
  *out = hh;
  return KSCF_OK;
}

extern "C" int kscf_ham_grid_info(const kscf_ham* ham, kscf_grid_info* info) {
  if (!ham || !info) {
    set_error("kscf_ham_grid_info: null argument");
    return KSCF_ERR_INVALID;
  }
  grid_info(ham->h.grid, info);
  return KSCF_OK;
}

extern "C" int kscf_set_potential(kscf_ham* ham, const double* v_slots, void* stream) {
  if (!ham || !v_slots) {
    set_error("kscf_set_potential: null argument");
    return KSCF_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  KSCF_CUDA_TRY(launch_mask_v(ham->h, v_slots, ham->h.d_v64, st));
  KSCF_CUDA_TRY(launch_v_to_f32(ham->h, st));
  return KSCF_OK;
}

extern "C" int kscf_get_potential(const kscf_ham* ham, double* v_slots, void* stream) {
  if (!ham || !v_slots) {
    set_error("kscf_get_potential: null argument");
    return KSCF_ERR_INVALID;
  }
  KSCF_CUDA_TRY(cudaMemcpyAsync(v_slots, ham->h.d_v64, sizeof(double) * ham->h.grid.n_slots,
                                cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return KSCF_OK;
}

extern "C" int kscf_spectral_bounds(const kscf_ham* ham, double* lower, double* upper) {
  if (!ham || !lower || !upper) {
    set_error("kscf_spectral_bounds: null argument");
    return KSCF_ERR_INVALID;
  }
  const Ham& H = ham->h;
  double* d2 = nullptr;
  KSCF_CUDA_TRY(cudaMalloc((void**)&d2, 2 * sizeof(double)));
  double mm[2] = {0, 0};
  cudaError_t e = launch_minmax_v(H, d2, 0);
  if (e == cudaSuccess) e = cudaMemcpy(mm, d2, 2 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d2);
  if (e != cudaSuccess) {
    kscf::set_error("kscf_spectral_bounds: %s", cudaGetErrorString(e));
    return KSCF_ERR_CUDA;
  }
  double sumabs = std::fabs(kW12[0]);
  for (int k = 1; k <= 6; k++) sumabs += 2.0 * std::fabs(kW12[k]);
  const double h = H.grid.h;
  *upper = 3.0 / (2.0 * h * h) * sumabs + mm[1] + H.kb_upper;
  *lower = mm[0] - H.kb_lower;
  return KSCF_OK;
}
