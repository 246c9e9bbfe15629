// Saving and loading a preconditioner set-up (the paper's reuse argument, Sections 1, 6.3 and 7.4: the
// set-up is paid once and serves further load cases and later runs).
//
// The file holds everything hplmm_setup computes from the assembled system -- decomposition and maps,
// mortars, the local factors and their layouts, the basis panels, the coarse factor and its launch
// schedules, the tuner's plans -- as named records (name, element size, count, bytes), after a header with
// a format tag, the options that shape the set-up and a fingerprint of the assembled system.  Loading
// requires a context assembled on the same system with the same set-up options; it restores every record by
// name, reallocates the work vectors and marks the context set up, so that apply and solve give the same
// results as on the context that was saved.  Device buffers move through a bounded host staging buffer.
#include "common.cuh"

#include <cstdio>
#include <cstring>
#include <map>

namespace hp {
namespace {

constexpr char MAGIC[8] = {'H', 'P', 'L', 'M', 'M', 'S', 'U', '1'};
constexpr size_t STAGE_BYTES = 256u << 20;

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

void put(FILE *f, const void *p, size_t bytes) {
  HP_REQUIRE(bytes == 0 || fwrite(p, 1, bytes, f) == bytes, HPLMM_ERR_INVALID, "save_setup: write failed");
}
void get(FILE *f, void *p, size_t bytes) {
  HP_REQUIRE(bytes == 0 || fread(p, 1, bytes, f) == bytes, HPLMM_ERR_INVALID,
             "load_setup: the file ends early or cannot be read");
}

// the options that shape the set-up (the others only steer how it runs)
struct SetupKey {
  int n_mortar, contact_halfwidth, n_st, local_prec, apply_prec, strict_two_grain, basis_solver, mortar_kind;
  int smoother_kind, pad_;
  double beta;
  int nx, ny, nz, n_nodes;
  long long n_dof, nnzb;
};

SetupKey key_of(const hplmm_ctx *c) {
  SetupKey k;
  std::memset(&k, 0, sizeof(k));
  k.n_mortar = c->opt.n_mortar;
  k.contact_halfwidth = c->opt.contact_halfwidth;
  k.n_st = c->opt.n_st;
  k.local_prec = c->opt.local_prec;
  k.apply_prec = c->opt.apply_prec;
  k.strict_two_grain = c->opt.strict_two_grain;
  k.basis_solver = c->opt.basis_solver;
  k.mortar_kind = c->opt.mortar_kind;
  k.smoother_kind = c->opt.smoother_kind;
  k.beta = c->opt.beta;
  k.nx = c->nx;
  k.ny = c->ny;
  k.nz = c->nz;
  k.n_nodes = c->n_nodes;
  k.n_dof = c->n_dof;
  k.nnzb = c->nnzb;
  return k;
}

// ---- record writer and reader (one visitor, two directions)
struct Saver {
  FILE *f;
  cudaStream_t s;
  std::vector<unsigned char> stage;
  void head(const std::string &name, size_t esz, unsigned long long count) {
    const unsigned nl = (unsigned)name.size();
    put(f, &nl, sizeof(nl));
    put(f, name.data(), nl);
    const unsigned long long e = esz;
    put(f, &e, sizeof(e));
    put(f, &count, sizeof(count));
  }
  template <typename T> void scalar(const std::string &name, T &v) {
    head(name, sizeof(T), 1);
    put(f, &v, sizeof(T));
  }
  template <typename T> void vec(const std::string &name, std::vector<T> &v) {
    head(name, sizeof(T), v.size());
    put(f, v.data(), v.size() * sizeof(T));
  }
  void vecvec(const std::string &name, std::vector<std::vector<int>> &v) {
    std::vector<long long> off(1, 0);
    std::vector<int> flat;
    for (auto &x : v) {
      flat.insert(flat.end(), x.begin(), x.end());
      off.push_back((long long)flat.size());
    }
    vec(name + ".off", off);
    vec(name + ".val", flat);
  }
  void launches(const std::string &name, std::vector<std::vector<FLaunch>> &v) {
    std::vector<long long> off(1, 0);
    std::vector<FLaunch> flat;
    for (auto &x : v) {
      flat.insert(flat.end(), x.begin(), x.end());
      off.push_back((long long)flat.size());
    }
    vec(name + ".off", off);
    vec(name + ".val", flat);
  }
  template <typename T> void buf(const std::string &name, Buf<T> &b) {
    const unsigned long long count = b.p ? b.n : 0;
    head(name, sizeof(T), count);
    const size_t total = count * sizeof(T);
    if (stage.size() < std::min(total, STAGE_BYTES)) stage.resize(std::min(total, STAGE_BYTES));
    for (size_t o = 0; o < total; o += STAGE_BYTES) {
      const size_t n = std::min(STAGE_BYTES, total - o);
      HP_CUDA(cudaMemcpyAsync(stage.data(), reinterpret_cast<const unsigned char *>(b.p) + o, n,
                              cudaMemcpyDeviceToHost, s));
      HP_CUDA(cudaStreamSynchronize(s));
      put(f, stage.data(), n);
    }
  }
};

struct Loader {
  FILE *f;
  cudaStream_t s;
  struct Rec {
    unsigned long long esz, count;
    long long pos;
  };
  std::map<std::string, Rec> idx;
  std::vector<unsigned char> stage;
  void index() {
    for (;;) {
      unsigned nl = 0;
      if (fread(&nl, 1, sizeof(nl), f) != sizeof(nl)) break;
      HP_REQUIRE(nl > 0 && nl < 256, HPLMM_ERR_INVALID, "load_setup: corrupt record header");
      std::string name(nl, '\0');
      get(f, &name[0], nl);
      Rec r;
      get(f, &r.esz, sizeof(r.esz));
      get(f, &r.count, sizeof(r.count));
      r.pos = ftell(f);
      idx[name] = r;
      HP_REQUIRE(fseek(f, (long)(r.esz * r.count), SEEK_CUR) == 0, HPLMM_ERR_INVALID, "load_setup: corrupt file");
    }
  }
  const Rec &find(const std::string &name, size_t esz) {
    auto it = idx.find(name);
    HP_REQUIRE(it != idx.end(), HPLMM_ERR_INVALID, "load_setup: record " + name + " is missing");
    HP_REQUIRE(it->second.esz == esz, HPLMM_ERR_INVALID, "load_setup: record " + name + " has another type");
    HP_REQUIRE(fseek(f, (long)it->second.pos, SEEK_SET) == 0, HPLMM_ERR_INVALID, "load_setup: seek failed");
    return it->second;
  }
  template <typename T> void scalar(const std::string &name, T &v) {
    const Rec &r = find(name, sizeof(T));
    HP_REQUIRE(r.count == 1, HPLMM_ERR_INVALID, "load_setup: record " + name + " is not a scalar");
    get(f, &v, sizeof(T));
  }
  template <typename T> void vec(const std::string &name, std::vector<T> &v) {
    const Rec &r = find(name, sizeof(T));
    v.resize(r.count);
    get(f, v.data(), r.count * sizeof(T));
  }
  void vecvec(const std::string &name, std::vector<std::vector<int>> &v) {
    std::vector<long long> off;
    std::vector<int> flat;
    vec(name + ".off", off);
    vec(name + ".val", flat);
    v.assign(off.empty() ? 0 : off.size() - 1, {});
    for (size_t i = 0; i + 1 < off.size(); ++i) v[i].assign(flat.begin() + off[i], flat.begin() + off[i + 1]);
  }
  void launches(const std::string &name, std::vector<std::vector<FLaunch>> &v) {
    std::vector<long long> off;
    std::vector<FLaunch> flat;
    vec(name + ".off", off);
    vec(name + ".val", flat);
    v.assign(off.empty() ? 0 : off.size() - 1, {});
    for (size_t i = 0; i + 1 < off.size(); ++i) v[i].assign(flat.begin() + off[i], flat.begin() + off[i + 1]);
  }
  template <typename T> void buf(const std::string &name, Buf<T> &b) {
    const Rec &r = find(name, sizeof(T));
    if (r.count == 0) {
      b.release();
      return;
    }
    b.alloc(r.count);
    const size_t total = r.count * sizeof(T);
    if (stage.size() < std::min(total, STAGE_BYTES)) stage.resize(std::min(total, STAGE_BYTES));
    for (size_t o = 0; o < total; o += STAGE_BYTES) {
      const size_t n = std::min(STAGE_BYTES, total - o);
      get(f, stage.data(), n);
      HP_CUDA(cudaMemcpyAsync(reinterpret_cast<unsigned char *>(b.p) + o, stage.data(), n, cudaMemcpyHostToDevice, s));
      HP_CUDA(cudaStreamSynchronize(s));
    }
  }
};

// ---- every field the set-up computes, by name
template <typename V> void visit_set(V &v, const std::string &pre, LocalSet &S) {
  v.scalar(pre + "count", S.count);
  v.vec(pre + "h_n", S.h_n);
  v.vec(pre + "h_bw", S.h_bw);
  v.vec(pre + "h_band_off", S.h_band_off);
  v.vec(pre + "h_node_off", S.h_node_off);
  v.vec(pre + "h_vec_off", S.h_vec_off);
  v.scalar(pre + "band_total", S.band_total);
  v.scalar(pre + "node_total", S.node_total);
  v.scalar(pre + "vec_total", S.vec_total);
  v.buf(pre + "box", S.box);
  v.buf(pre + "n", S.n);
  v.buf(pre + "bw", S.bw);
  v.buf(pre + "band_off", S.band_off);
  v.buf(pre + "node_off", S.node_off);
  v.buf(pre + "vec_off", S.vec_off);
  v.buf(pre + "lnodes", S.lnodes);
  v.buf(pre + "lmap", S.lmap);
  v.buf(pre + "band64", S.band64);
  v.buf(pre + "band32", S.band32);
  v.buf(pre + "band16", S.band16);
  v.scalar(pre + "apply_bf16", S.apply_bf16);
  v.buf(pre + "order", S.order);
  v.buf(pre + "queue", S.queue);
  v.buf(pre + "gidx", S.gidx);
  v.buf(pre + "yscr", S.yscr);
  v.scalar(pre + "tuned_chunk_rows", S.tuned_chunk_rows);
  v.scalar(pre + "tuned_ring_rows", S.tuned_ring_rows);
  v.scalar(pre + "tuned_c0_stages", S.tuned_c0_stages);
  v.scalar(pre + "tuned_cluster", S.tuned_cluster);
  v.scalar(pre + "tuned_bulk", S.tuned_bulk);
  v.scalar(pre + "prec", S.prec);
}

template <typename V> void visit_cf(V &v, CoarseFactor &F) {
  v.scalar("cf.nf", F.nf);
  v.scalar("cf.nlev", F.nlev);
  v.scalar("cf.F_total", F.F_total);
  v.scalar("cf.Y_total", F.Y_total);
  v.scalar("cf.D_total", F.D_total);
  v.scalar("cf.idx_total", F.idx_total);
  v.vec("cf.h_m", F.h_m);
  v.vec("cf.h_P", F.h_P);
  v.vec("cf.h_p", F.h_p);
  v.vec("cf.h_b", F.h_b);
  v.vec("cf.h_parent", F.h_parent);
  v.vec("cf.h_level", F.h_level);
  v.vec("cf.h_foff", F.h_foff);
  v.vec("cf.h_yoff", F.h_yoff);
  v.vec("cf.h_doff", F.h_doff);
  v.vec("cf.h_ioff", F.h_ioff);
  v.buf("cf.m", F.m);
  v.buf("cf.P", F.P);
  v.buf("cf.p", F.p);
  v.buf("cf.b", F.b);
  v.buf("cf.parent", F.parent);
  v.buf("cf.foff", F.foff);
  v.buf("cf.yoff", F.yoff);
  v.buf("cf.doff", F.doff);
  v.buf("cf.ioff", F.ioff);
  v.buf("cf.roff", F.roff);
  v.buf("cf.idx", F.idx);
  v.buf("cf.rank", F.rank);
  v.buf("cf.rel", F.rel);
  v.buf("cf.erank", F.erank);
  v.buf("cf.owner", F.owner);
  v.buf("cf.fpos", F.fpos);
  v.buf("cf.F", F.F);
  v.buf("cf.Y", F.Y);
  v.buf("cf.D", F.D);
  v.buf("cf.tasks", F.tasks);
  v.buf("cf.otask", F.otask);
  v.buf("cf.oz_S", F.oz_S);
  v.buf("cf.oz_E", F.oz_E);
  v.scalar("cf.oz_slots", F.oz_slots);
  v.vec("cf.fact", F.fact);
  v.launches("cf.fwd", F.fwd);
  v.launches("cf.bwd", F.bwd);
  v.scalar("cf.flops", F.flops);
  v.scalar("cf.solve_bytes", F.solve_bytes);
}

template <typename V> void visit_ctx(V &v, hplmm_ctx *c) {
  // decomposition and maps
  v.scalar("n_grains", c->n_grains);
  v.scalar("px", c->px);
  v.scalar("py", c->py);
  v.scalar("pz", c->pz);
  v.scalar("n_ifaces", c->n_ifaces);
  v.scalar("n_iface_nodes", c->n_iface_nodes);
  v.buf("vgrain", c->vgrain);
  v.buf("node_cls", c->node_cls);
  v.buf("iface_of_node", c->iface_of_node);
  v.buf("iface_slot", c->iface_slot);
  v.buf("iface_pair", c->iface_pair);
  v.buf("iface_off", c->iface_off);
  v.buf("iface_nodes", c->iface_nodes);
  v.vec("h_iface_off", c->h_iface_off);
  v.vec("h_gi_off", c->h_gi_off);
  v.vec("h_gi_iface", c->h_gi_iface);
  v.vec("h_gi_colbase", c->h_gi_colbase);
  v.buf("gi_off", c->gi_off);
  v.buf("gi_iface", c->gi_iface);
  v.buf("gi_colbase", c->gi_colbase);
  v.vec("h_kg", c->h_kg);
  v.vec("h_panel_off", c->h_panel_off);
  v.buf("kg", c->kg);
  v.buf("panel_off", c->panel_off);
  v.vec("h_corr_col", c->h_corr_col);
  v.vecvec("h_glists", c->h_glists);
  v.vec("h_grain_hasb", c->h_grain_hasb);
  v.buf("corr_col", c->corr_col);
  v.buf("b_corr", c->b_corr);
  // mortars
  v.scalar("n_mortars", c->n_mortars);
  v.buf("mortar_off", c->mortar_off);
  v.buf("mortar_nodes", c->mortar_nodes);
  v.buf("mortar_idx", c->mortar_idx);
  v.buf("eta_off", c->eta_off);
  v.buf("eta", c->eta);
  v.buf("comp_mask", c->comp_mask);
  v.buf("col_off", c->col_off);
  v.vec("h_mortar_off", c->h_mortar_off);
  v.vec("h_comp_mask", c->h_comp_mask);
  v.vec("h_col_off", c->h_col_off);
  v.scalar("n_mortar_cols", c->n_mortar_cols);
  v.scalar("n_coarse", c->n_coarse);
  // local problems and the algebraic mortars' interface data
  visit_set(v, "grains.", c->grains);
  visit_set(v, "contacts.", c->contacts);
  v.buf("mslot_of_node", c->mslot_of_node);
  v.buf("mfree", c->mfree);
  v.buf("mcol", c->mcol);
  v.buf("qblk", c->qblk);
  v.buf("qoff", c->qoff);
  // coarse space
  v.buf("X64", c->X64);
  v.buf("X32", c->X32);
  v.buf("X16", c->X16);
  v.buf("panel_off_cm", c->panel_off_cm);
  v.vec("h_panel_off_cm", c->h_panel_off_cm);
  v.scalar("dense_ao", c->dense_ao);
  v.buf("Ao", c->Ao);
  visit_cf(v, c->cf);
  v.buf("gcol_off", c->gcol_off);
  v.buf("gcol", c->gcol);
  v.scalar("t_ml", c->t_ml);
  v.scalar("t_mg", c->t_mg);
}

}  // namespace

void save_setup(hplmm_ctx *c, const char *path) {
  HP_REQUIRE(path && *path, HPLMM_ERR_INVALID, "save_setup: no path");
  HP_CUDA(cudaStreamSynchronize(c->stream));
  File fh;
  fh.f = fopen(path, "wb");
  HP_REQUIRE(fh.f != nullptr, HPLMM_ERR_INVALID, std::string("save_setup: cannot open ") + path);
  put(fh.f, MAGIC, sizeof(MAGIC));
  SetupKey k = key_of(c);
  put(fh.f, &k, sizeof(k));
  Saver sv{fh.f, c->stream, {}};
  visit_ctx(sv, c);
  HP_REQUIRE(fflush(fh.f) == 0, HPLMM_ERR_INVALID, "save_setup: write failed");
}

void load_setup(hplmm_ctx *c, const char *path) {
  HP_REQUIRE(path && *path, HPLMM_ERR_INVALID, "load_setup: no path");
  File fh;
  fh.f = fopen(path, "rb");
  HP_REQUIRE(fh.f != nullptr, HPLMM_ERR_INVALID, std::string("load_setup: cannot open ") + path);
  char magic[sizeof(MAGIC)];
  get(fh.f, magic, sizeof(magic));
  HP_REQUIRE(std::memcmp(magic, MAGIC, sizeof(MAGIC)) == 0, HPLMM_ERR_INVALID,
             "load_setup: not a saved set-up of this format");
  SetupKey k, mine = key_of(c);
  get(fh.f, &k, sizeof(k));
  HP_REQUIRE(std::memcmp(&k, &mine, sizeof(k)) == 0, HPLMM_ERR_INVALID,
             "load_setup: the file was saved for another system or other set-up options (image, n_mortar, "
             "beta, contact_halfwidth, n_st, precisions, basis solver, mortar kind, smoother kind must match)");
  c->setup_done = false;
  drop_apply_graph(c);
  Loader ld{fh.f, c->stream, {}, {}};
  ld.index();
  visit_ctx(ld, c);
  c->status.alloc(4);  // the device error word (the set-up allocates it with the maps)
  c->status.zero(c->stream);
  HP_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace hp
