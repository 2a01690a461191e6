// io.cu - hb_save / hb_load: the compressed operator as a file (host code).
//
// Layout (little-endian; every integer int64, every real double; see
// include/hb.h for the meaning of each field):
//   "HBFACT01"
//   nx ny | x0 y0 h omega | eps chi nbr_radius_h | leaf precision workspace_mb barrier_cycles
//   n_I | nodes_x[n_I] nodes_y[n_I] | tau2[N_I^2] v0[N_I^2] v1[N_I^2] | n_cells[N_v]
//   L_v | perm[N_v] | bounds of levels 0..L_v (2^l + 1 each)
//   n_factor | arena[2 n_factor] (complex128: re, im)
//   leaf_off[2^L_v]
//   n_butterfly | per butterfly: l oi si L | (rank, f_off) for k = 0..L, block 0..2^L-1 | kl_off[2^L]
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

namespace {

const char kMagic[8] = {'H', 'B', 'F', 'A', 'C', 'T', '0', '1'};

struct File {
  FILE* f = nullptr;
  std::string path;
  long long size = -1;   // bytes in the file (reading); -1: unknown
  ~File() {
    if (f) fclose(f);
  }
};

// Bytes left to read; a count read from the file is checked against it
// before anything is allocated for it.
long long remaining(File& F) {
  if (F.size < 0) return -1;
  const long pos = ftell(F.f);
  return pos < 0 ? -1 : F.size - (long long)pos;
}

void need(File& F, long long count, size_t elem) {
  const long long left = remaining(F);
  if (count < 0 || (left >= 0 && (unsigned long long)count > (unsigned long long)left / elem))
    throw Error{HB_ERR_ARG, "truncated or corrupt factor file " + F.path};
}

void put_raw(File& F, const void* p, size_t bytes) {
  if (bytes && fwrite(p, 1, bytes, F.f) != bytes)
    throw Error{HB_ERR_ARG, "cannot write " + F.path};
}
void put_i(File& F, long long v) { put_raw(F, &v, sizeof v); }
void put_d(File& F, double v) { put_raw(F, &v, sizeof v); }
template <class T>
void put_vec(File& F, const std::vector<T>& v) {
  put_raw(F, v.data(), v.size() * sizeof(T));
}

void get_raw(File& F, void* p, size_t bytes) {
  if (bytes && fread(p, 1, bytes, F.f) != bytes)
    throw Error{HB_ERR_ARG, "truncated or unreadable factor file " + F.path};
}
long long get_i(File& F) {
  long long v;
  get_raw(F, &v, sizeof v);
  return v;
}
double get_d(File& F) {
  double v;
  get_raw(F, &v, sizeof v);
  return v;
}
long long get_count(File& F, long long lo, long long hi, const char* what) {
  const long long v = get_i(F);
  if (v < lo || v > hi) throw Error{HB_ERR_ARG, std::string("factor file: bad ") + what};
  return v;
}
template <class T>
std::vector<T> get_vec(File& F, long long n) {
  need(F, n, sizeof(T));
  std::vector<T> v((size_t)n);
  get_raw(F, v.data(), (size_t)n * sizeof(T));
  return v;
}

}  // namespace

void save_file(const hb_ctx* c, const char* path) {
  File F;
  F.path = path;
  F.f = fopen(path, "wb");
  if (!F.f) throw Error{HB_ERR_ARG, std::string("cannot open ") + path + " for writing"};
  put_raw(F, kMagic, sizeof kMagic);
  put_i(F, c->nx);
  put_i(F, c->ny);
  put_d(F, c->x0);
  put_d(F, c->y0);
  put_d(F, c->h);
  put_d(F, c->omega);
  put_d(F, c->opt.eps);
  put_d(F, c->opt.chi);
  put_d(F, c->opt.nbr_radius_h);
  put_i(F, c->opt.leaf);
  put_i(F, c->opt.precision);
  put_i(F, c->opt.workspace_mb);
  put_i(F, c->opt.barrier_cycles);
  put_i(F, c->nI);
  put_vec(F, c->nodes_x);
  put_vec(F, c->nodes_y);
  for (int q = 0; q < 3; ++q) put_vec(F, c->tab[q]);
  put_vec(F, c->n_cells);
  put_i(F, c->Lv);
  put_vec(F, c->perm);
  for (int l = 0; l <= c->Lv; ++l) put_vec(F, c->bounds[(size_t)l]);
  put_i(F, c->n_factor);
  {
    // the arena in slices of 64 Mi entries
    const long long slice = 1LL << 26;
    std::vector<double2> h((size_t)std::min(c->n_factor, slice));
    for (long long o = 0; o < c->n_factor; o += slice) {
      const long long m = std::min(slice, c->n_factor - o);
      HB_CUDA(cudaMemcpy(h.data(), c->d_f64 + o, (size_t)m * sizeof(double2), cudaMemcpyDeviceToHost));
      put_raw(F, h.data(), (size_t)m * sizeof(double2));
    }
  }
  put_vec(F, c->leaf_off);
  put_i(F, (long long)c->bidx.size());
  for (const BflyIndex& b : c->bidx) {
    put_i(F, b.l);
    put_i(F, b.oi);
    put_i(F, b.si);
    put_i(F, b.L);
    for (int k = 0; k <= b.L; ++k)
      for (size_t j = 0; j < b.rank[(size_t)k].size(); ++j) {
        put_i(F, b.rank[(size_t)k][j]);
        put_i(F, b.f_off[(size_t)k][j]);
      }
    put_vec(F, b.kl_off);
  }
  if (fflush(F.f) != 0) throw Error{HB_ERR_ARG, std::string("cannot write ") + path};
}

hb_ctx* load_file(const char* path,
                  hb_ctx* (*create)(const hb_grid*, const hb_tables*, double, const hb_options*)) {
  File F;
  F.path = path;
  F.f = fopen(path, "rb");
  if (!F.f) throw Error{HB_ERR_ARG, std::string("cannot open ") + path};
  if (fseek(F.f, 0, SEEK_END) == 0) {
    const long end = ftell(F.f);
    F.size = end < 0 ? -1 : (long long)end;
  }
  if (fseek(F.f, 0, SEEK_SET) != 0) throw Error{HB_ERR_ARG, std::string("cannot read ") + path};
  char magic[8];
  get_raw(F, magic, sizeof magic);
  if (std::memcmp(magic, kMagic, sizeof magic) != 0) throw Error{HB_ERR_ARG, "not an HB factor file"};
  hb_grid g{};
  g.nx = (int)get_count(F, 1, 1LL << 31, "nx");
  g.ny = (int)get_count(F, 1, 1LL << 31, "ny");
  g.x0 = get_d(F);
  g.y0 = get_d(F);
  g.h = get_d(F);
  const double omega = get_d(F);
  hb_options o{};
  o.eps = get_d(F);
  o.chi = get_d(F);
  o.nbr_radius_h = get_d(F);
  o.leaf = (int)get_count(F, 1, 1LL << 31, "leaf");
  o.precision = (int)get_i(F);
  o.workspace_mb = (int)get_i(F);
  o.barrier_cycles = get_i(F);
  const long long nI = get_count(F, 2, 16, "n_I");
  const long long NI = nI * nI;
  const long long Nv = (long long)g.nx * g.ny;
  std::vector<double> nx_ = get_vec<double>(F, nI), ny_ = get_vec<double>(F, nI);
  std::vector<double> tab[3];
  for (int q = 0; q < 3; ++q) tab[q] = get_vec<double>(F, NI * NI);
  std::vector<double> ncell = get_vec<double>(F, Nv);
  hb_tables t{};
  t.n_I = (int)nI;
  t.nodes_x = nx_.data();
  t.nodes_y = ny_.data();
  t.tau2 = tab[0].data();
  t.v0 = tab[1].data();
  t.v1 = tab[2].data();
  t.n_cells = ncell.data();
  hb_ctx* c = create(&g, &t, omega, &o);   // validates, uploads the tables, builds the tree
  std::unique_ptr<hb_ctx, void (*)(hb_ctx*)> guard(c, [](hb_ctx* p) { hb_destroy(p); });
  // the tree is a function of the grid and the leaf size: the file must agree
  if (get_i(F) != c->Lv) throw Error{HB_ERR_ARG, "factor file: tree depth differs from its grid"};
  if (get_vec<long long>(F, Nv) != c->perm) throw Error{HB_ERR_ARG, "factor file: tree order differs"};
  for (int l = 0; l <= c->Lv; ++l)
    if (get_vec<long long>(F, (1LL << l) + 1) != c->bounds[(size_t)l])
      throw Error{HB_ERR_ARG, "factor file: tree nodes differ"};
  c->n_factor = get_count(F, 0, 1LL << 40, "arena size");
  need(F, c->n_factor, sizeof(double2));
  c->d_f64 = dev_alloc<double2>((size_t)c->n_factor + 16);
  HB_CUDA(cudaMemset(c->d_f64, 0, sizeof(double2) * ((size_t)c->n_factor + 16)));
  {
    const long long slice = 1LL << 26;
    std::vector<double2> h((size_t)std::min(c->n_factor, slice));
    for (long long off = 0; off < c->n_factor; off += slice) {
      const long long m = std::min(slice, c->n_factor - off);
      get_raw(F, h.data(), (size_t)m * sizeof(double2));
      HB_CUDA(cudaMemcpy(c->d_f64 + off, h.data(), (size_t)m * sizeof(double2), cudaMemcpyHostToDevice));
    }
  }
  auto leaf_size = [&](long long t) { return c->bounds[(size_t)c->Lv][(size_t)t + 1] - c->bounds[(size_t)c->Lv][(size_t)t]; };
  auto in_arena = [&](long long off, long long n) {
    if (off < 0 || n < 0 || off + n > c->n_factor) throw Error{HB_ERR_ARG, "factor file: block outside the arena"};
  };
  c->leaf_off = get_vec<long long>(F, 1LL << c->Lv);
  for (long long t = 0; t < (1LL << c->Lv); ++t) in_arena(c->leaf_off[(size_t)t], leaf_size(t) * leaf_size(t));
  // the butterflies in HODBF order: level l = 1..L_v, sibling pair p, (2p, 2p + 1) then (2p + 1, 2p)
  std::vector<int> want_l, want_oi, want_si;
  for (int l = 1; l <= c->Lv; ++l)
    for (long long p = 0; p < (1LL << (l - 1)); ++p)
      for (int d = 0; d < 2; ++d) {
        want_l.push_back(l);
        want_oi.push_back((int)(2 * p + d));
        want_si.push_back((int)(2 * p + 1 - d));
      }
  const long long nb = get_count(F, 0, 1LL << 31, "butterfly count");
  if (nb != (long long)want_l.size()) throw Error{HB_ERR_ARG, "factor file: wrong number of butterflies"};
  for (long long q = 0; q < nb; ++q) {
    BflyIndex b;
    b.l = (int)get_i(F);
    b.oi = (int)get_i(F);
    b.si = (int)get_i(F);
    if (b.l != want_l[(size_t)q] || b.oi != want_oi[(size_t)q] || b.si != want_si[(size_t)q])
      throw Error{HB_ERR_ARG, "factor file: butterflies out of HODBF order"};
    b.L = (int)get_count(F, c->Lv - b.l, c->Lv - b.l, "butterfly levels");
    b.rank.assign((size_t)b.L + 1, {});
    b.f_off.assign((size_t)b.L + 1, {});
    for (int k = 0; k <= b.L; ++k)
      for (long long j = 0; j < (1LL << b.L); ++j) {
        b.rank[(size_t)k].push_back((int)get_count(F, 0, 1 << 20, "rank"));
        b.f_off[(size_t)k].push_back(get_i(F));
      }
    b.kl_off = get_vec<long long>(F, 1LL << b.L);
    // every block inside the arena
    const long long w0 = 1LL << b.L;
    for (long long j = 0; j < w0; ++j) {
      const long long leaf = ((long long)b.si << b.L) + j;
      in_arena(b.f_off[0][(size_t)j], (long long)b.rank[0][(size_t)j] * leaf_size(leaf));
    }
    for (int k = 1; k <= b.L; ++k) {
      const long long w = 1LL << (b.L - k);
      for (long long i = 0; i < (1LL << k); ++i)
        for (long long j = 0; j < w; ++j) {
          const size_t q1 = (size_t)((i / 2) * (2 * w) + 2 * j);
          const long long cols = (long long)b.rank[(size_t)k - 1][q1] + b.rank[(size_t)k - 1][q1 + 1];
          in_arena(b.f_off[(size_t)k][(size_t)(i * w + j)], (long long)b.rank[(size_t)k][(size_t)(i * w + j)] * cols);
        }
    }
    for (long long i = 0; i < w0; ++i) {
      const long long leaf = ((long long)b.oi << b.L) + i;
      in_arena(b.kl_off[(size_t)i], leaf_size(leaf) * b.rank[(size_t)b.L][(size_t)i]);
    }
    c->bidx.push_back(std::move(b));
  }
  plans_from_index(c);
  c->built = true;
  return guard.release();
}

}  // namespace hb
