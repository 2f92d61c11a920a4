// C ABI of libfmg_eig: level hierarchy, the full multigrid scheme (Algorithm 3.2) as one
// CUDA graph per handle, batches of independent instances, and the component entry points
// used to check each step.
//
// A handle holds a batch of nb instances (nb = 1 for fmg_eig_create) sorted by level count,
// largest first.  Level k's arrays hold the cnt[k] instances that have a level k back to
// back, so on the FMG stage of level k the active instances are 0 .. cnt[k] - 1 of every
// array and each step of the stage is one launch over all of them (Grid::nb).
#include <atomic>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "engine.h"

using namespace fmg;

namespace fmg {

Level view(const Level& l, int first, int count) {
  Level v = l;
  const size_t o = (size_t)first * l.g.stride;
  auto adv = [o](auto*& p) {
    if (p) p += o;
  };
  adv(v.c.cC); adv(v.c.cE); adv(v.c.cN); adv(v.c.cNE); adv(v.c.dinv);
  adv(v.cw.cC); adv(v.cw.cE); adv(v.cw.cN); adv(v.cw.cNE); adv(v.cw.dinv);
  adv(v.cw3.dinv);
  for (int q = 0; q < 8; ++q) {
    adv(v.cw3.a[q]);
    adv(v.c3.a[q]);
    adv(v.b3.a[q]);
  }
  adv(v.c3.dinv);
  adv(v.x); adv(v.xt); adv(v.f); adv(v.r); adv(v.u); adv(v.y); adv(v.z);
  adv(v.b.C); adv(v.b.E); adv(v.b.N); adv(v.b.NE);
  adv(v.x32); adv(v.xt32); adv(v.f32); adv(v.r32); adv(v.uhi); adv(v.ulo);
  v.c.tab = v.c3.tab = v.cw.tab = v.cw3.tab = nullptr;  // per-instance tables are not sliced
  v.ct = CoefT{};
  v.g.nb = count;
  return v;
}

}  // namespace fmg

namespace {

// ---- dimension dispatch of the level kernels -----------------------------------------------
void lv_coef(Level& l, const PotentialParams* p, cudaStream_t s, bool full = false) {
  if (l.g.dim == 2) coef2d_setup(l.g, p, full ? l.cw : l.c, s);
  else coef3d_setup(l.g, p, full ? l.cw3 : l.c3, s);
}
void lv_apply(Level& l, const double* x, double* y, cudaStream_t s) {
  if (l.g.dim == 2) apply2d(l.g, l.c, x, y, s);
  else apply3d(l.g, l.c3, x, y, s);
}
// y = (A + W) x, whatever the form of the auxiliary operator
void lv_apply_full(Level& l, const double* x, double* y, cudaStream_t s) {
  if (l.g.dim == 2) apply2d(l.g, l.cw, x, y, s);
  else apply3d(l.g, l.cw3, x, y, s);
}
// f -= W u (paper-literal form: W moves to the right-hand side)
void lv_sub_wmass(Level& l, const double* u, double* f, cudaStream_t s) {
  if (l.g.dim == 2) sub_wmass2d(l.g, l.cw, l.c, u, f, s);
  else sub_wmass3d(l.g, l.cw3, l.c3, u, f, s);
}
void lv_mass(Level& l, const double* x, double* y, cudaStream_t s) {
  if (l.g.dim == 2) mass2d(l.g, x, y, s);
  else mass3d(l.g, x, y, s);
}
void lv_mass_df(Level& l, SplitVec x, double* y, cudaStream_t s) {
  if (l.g.dim == 2) mass2d_df(l.g, x, y, s);
  else mass3d_df(l.g, x, y, s);
}
void lv_jacobi(Level& l, const double* f, const double* x, double* xo, bool zero, cudaStream_t s) {
  if (l.g.dim == 2) jacobi2d(l.g, l.c, f, x, xo, zero, s);
  else jacobi3d(l.g, l.c3, f, x, xo, zero, s);
}
void lv_cheb(Level& l, const double* f, const double* x, double* d, double* xo, double alpha,
             double beta, bool first, bool zero, cudaStream_t s) {
  if (l.g.dim == 2) cheb2d(l.g, l.c, f, x, d, xo, alpha, beta, first, zero, s);
  else cheb3d(l.g, l.c3, f, x, d, xo, alpha, beta, first, zero, s);
}
void lv_residual(Level& l, const double* f, const double* x, double* r, cudaStream_t s) {
  if (l.g.dim == 2) residual2d(l.g, l.c, f, x, r, s);
  else residual3d(l.g, l.c3, f, x, r, s);
}
void lv_restrict(Level& fl, Level& cl, const double* rf, double* rc, cudaStream_t s,
                 const double* rf2 = nullptr, double* rc2 = nullptr) {
  if (fl.g.dim == 2) restrict2d(fl.g, cl.g, rf, rc, s, rf2, rc2);
  else restrict3d(fl.g, cl.g, rf, rc, s, rf2, rc2);
}
void lv_prolong(Level& fl, Level& cl, const double* ec, double* xf, bool add, const double* extra,
                const double* scale, int scale_stride, cudaStream_t s) {
  if (fl.g.dim == 2) prolong2d(fl.g, cl.g, ec, xf, add, extra, scale, scale_stride, s);
  else prolong3d(fl.g, cl.g, ec, xf, add, extra, scale, scale_stride, s);
}
void lv_nload(Level& l, const double* u, double* out, cudaStream_t s) {
  if (l.g.dim == 2) nload2d(l.g, u, out, s);
  else nload3d(l.g, u, out, s);
}
void lv_rhs(Level& l, const double* lam, const PotentialParams* p, const double* u, double* f,
            cudaStream_t s) {
  if (l.g.dim == 2) rhs2d(l.g, lam, p, u, f, s);
  else rhs3d(l.g, lam, p, u, f, s);
}
void lv_rhs_f32(Level& l, const double* lam, const PotentialParams* p, const double* u,
                double* f, cudaStream_t s) {
  if (l.g.dim == 2) rhs2d_f32(l.g, lam, p, u, f, s);
  else rhs3d_f32(l.g, lam, p, u, f, s);
}
void lv_nload_density(Level& l, const double* u, double* nl, cudaStream_t s) {
  if (l.g.dim == 2) nload_density2d(l.g, u, nl, l.b, s);
  else nload_density3d(l.g, u, nl, l.b3, s);
}
// Mixed-precision modes: the nonlinear kernels compute in double-float arithmetic from the
// split of u into l.uhi + l.ulo (written here, on the same stream, just before).
SplitVec lv_split(Level& l, const double* u, cudaStream_t s) {
  split_df(u, l.uhi, l.ulo, l.g.stride * l.g.nb, s);
  return SplitVec{l.uhi, l.ulo};
}
void lv_rhs_df(Level& l, const double* lam, const PotentialParams* p, const double* u, double* f,
               cudaStream_t s) {
  const SplitVec v = lv_split(l, u, s);
  if (l.g.dim == 2) rhs2d_df(l.g, lam, p, v, f, s);
  else rhs3d_df(l.g, lam, p, v, f, s);
}
void lv_nload_density_df(Level& l, SplitVec v, double* nl, cudaStream_t s) {
  if (l.g.dim == 2) nload_density2d_df(l.g, v, nl, l.b, s);
  else nload_density3d_df(l.g, v, nl, l.b3, s);
}
// split: the density stencils hold double-float splits (mixed modes, from the _df kernels)
void lv_coarsen_density(Level& fl, Level& cl, cudaStream_t s, bool split) {
  if (fl.g.dim == 2) coarsen_density2d(fl.g, cl.g, fl.b, cl.b, s, split);
  else coarsen_density3d(fl.g, cl.g, fl.b3, cl.b3, s, split);
}
void lv_t3(Level& l, int n1, const double* u, double* partials, double* t3, cudaStream_t s) {
  if (l.g.dim == 2) t3_moments2d(l.g, n1, u, l.pw, l.t3map, partials, t3, s);
  else t3_moments3d(l.g, n1, u, l.pw, l.t3map, partials, t3, s);
}
void lv_dense_level1(Level& l1, double* L, double* M, cudaStream_t s, bool full) {
  if (l1.g.dim == 2) dense_level1_2d(l1.g, full ? l1.cw : l1.c, L, M, s);
  else dense_level1_3d(l1.g, full ? l1.cw3 : l1.c3, L, M, s);
}
void lv_start(Level& l1, double* c, int cstride, cudaStream_t s) {
  if (l1.g.dim == 2) start_vector(l1.g, c, cstride, s);
  else start_vector3d(l1.g, c, cstride, s);
}
void lv_gather_level1(Level& l1, double* gA, double* gM, double* t1, double* B1, cudaStream_t s,
                      bool split) {
  if (l1.g.dim == 2) {
    gather_level1_2d(l1.g, l1.y, l1.z, l1.r, l1.b, gA, gM, t1, B1, s, split);
  } else {
    gather_vec3d(l1.g, l1.y, l1.z, l1.r, gA, gM, t1, s);
    density_dense3d(l1.g, l1.b3, B1, s, split);
  }
}

double factorial(int k) {
  double r = 1.0;
  for (int i = 2; i <= k; ++i) r *= i;
  return r;
}

}  // namespace

fmg_eig_handle::~fmg_eig_handle() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (ev_fork) cudaEventDestroy(ev_fork);
  for (StageMark& m : marks)
    if (m.ev) cudaEventDestroy(m.ev);
  for (cudaEvent_t e : ev_join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : ev_level)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < kProfCount; ++i)
    for (int j = 0; j < 2; ++j)
      if (prof[i][j]) cudaEventDestroy(prof[i][j]);
  for (void* p : allocs) {
    if (opt.async_alloc) cudaFreeAsync(p, stream);
    else cudaFree(p);
  }
  if (hparams) {
    if (opt.async_alloc) delete[] hparams;
    else cudaFreeHost(hparams);
  }
  for (cudaStream_t x : side)
    if (x) cudaStreamDestroy(x);
  if (stream) cudaStreamDestroy(stream);
}

namespace fmg {

#define CK(expr)                                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) {                         \
      return FMG_ECUDA;                              \
    }                                                \
  } while (0)

int validate(const fmg_eig_problem* p) {
  if (!p) return FMG_EINVAL;
  if (p->dim != 2 && p->dim != 3) return FMG_EINVAL;
  if (p->coarse_cells < 2 || p->levels < 1 || p->levels > FMG_MAX_LEVELS) return FMG_EINVAL;
  if (p->nu_pre < 0 || p->nu_post < 0 || p->vcycles < 1 || p->corrections < 1)
    return FMG_EINVAL;
  if (!(p->box_len > 0.0) || !(p->zeta >= 0.0) || !(p->omega > 0.0 && p->omega <= 1.0))
    return FMG_EINVAL;
  if (!(p->scf_tol > 0.0) || p->scf_max_iter < 1) return FMG_EINVAL;
  if (p->flags &
      ~(FMG_FLAG_NO_AUTOTUNE | FMG_FLAG_FP32_RHS | FMG_FLAG_NO_TMA | FMG_FLAG_STAR_WALKS |
        FMG_FLAG_SEPARATE_VCYCLE | FMG_FLAG_EXPIRE_WAITS))
    return FMG_EINVAL;
  if ((p->flags & FMG_FLAG_FP32_RHS) && p->precision == FMG_FP64) return FMG_EINVAL;
  const double cells = (double)p->coarse_cells * pow(2.0, p->levels - 1);
  if (cells > (p->dim == 2 ? 32768.0 : 1024.0)) return FMG_EINVAL;
  if (p->smoother != FMG_SMOOTH_JACOBI && p->smoother != FMG_SMOOTH_CHEBYSHEV &&
      p->smoother != FMG_SMOOTH_CG)
    return FMG_EINVAL;
  if (p->smoother != FMG_SMOOTH_JACOBI && p->precision != FMG_FP64) return FMG_ENOTSUP;
  if ((p->precision != FMG_FP64 && p->precision != FMG_MIXED_FP32 &&
       p->precision != FMG_MIXED_BF16) ||
      (p->operator_form != FMG_W_LEFT && p->operator_form != FMG_PAPER_LITERAL))
    return FMG_ENOTSUP;
  return FMG_OK;
}

// the fields every instance of a batch shares (all but levels and the PDE coefficients)
auto shared_key(const fmg_eig_problem& p) {
  return std::make_tuple(p.dim, p.coarse_cells, p.nu_pre, p.nu_post, p.vcycles, p.corrections,
                         p.smoother, p.precision, p.operator_form, p.scf_max_iter, p.flags,
                         p.box_len, p.scf_tol);
}

bool same_shared_settings(const fmg_eig_problem& a, const fmg_eig_problem& b) {
  return shared_key(a) == shared_key(b);
}

PotentialParams potential(const fmg_eig_problem& p) {
  PotentialParams q{};
  q.w0 = p.w_const;
  q.wx = p.w_quad[0];
  q.wy = p.w_quad[1];
  q.wz = p.w_quad[2];
  q.zeta = p.zeta;
  q.omega = p.smoother == FMG_SMOOTH_CHEBYSHEV ? 1.0 : p.omega;  // dinv = omega / D
  q.operator_form = p.operator_form;
  return q;
}

// host staging of every instance's parameters (and their W_LEFT copies, paper-literal form)
void fill_params(fmg_eig_handle* h) {
  for (int b = 0; b < h->nb; ++b) {
    h->hparams[b] = potential(h->probs[b]);
    if (h->literal()) {
      h->hparams[h->nb + b] = h->hparams[b];
      h->hparams[h->nb + b].operator_form = FMG_W_LEFT;
    }
  }
}

}  // namespace fmg

cudaError_t fmg::upload_params(fmg_eig_handle* h, cudaStream_t s) {
  return cudaMemcpyAsync(h->dparams, h->hparams, sizeof(PotentialParams) * h->nparams,
                         cudaMemcpyHostToDevice, s);
}

namespace fmg {

void build_levels(fmg_eig_handle* h) {
  const fmg_eig_problem& p = h->prob;
  const int dim = p.dim;
  h->lv.resize(p.levels);
  for (int k = 1; k <= p.levels; ++k) {
    Level& l = h->L(k);
    l.cap = h->cnt[k];
    l.g.dim = dim;
    l.g.n = p.coarse_cells << (k - 1);
    l.g.rows = l.g.n + 1;
    l.g.pitch = (l.g.n + 1 + 31) / 32 * 32;
    l.g.stride = (size_t)l.g.rows * l.g.pitch * (dim == 3 ? (size_t)l.g.rows : 1);
    l.g.h = p.box_len / l.g.n;
    l.g.nb = l.cap;
    l.g.walk_all = (p.flags & FMG_FLAG_STAR_WALKS) != 0;
    const size_t s = l.g.stride * l.cap;
    if (dim == 2) {
      l.c.cC = h->alloc<double>(s);
      l.c.cE = h->alloc<double>(s);
      l.c.cN = h->alloc<double>(s);
      l.c.cNE = h->alloc<double>(s);
      l.c.dinv = h->alloc<double>(s);
      l.c.tab = h->alloc<double>(8 * (size_t)(l.g.n + 1) * l.cap);
      l.b.C = h->alloc<double>(s);
      l.b.E = h->alloc<double>(s);
      l.b.N = h->alloc<double>(s);
      l.b.NE = h->alloc<double>(s);
      l.cw = l.c;
      if (h->literal()) {
        l.cw.cC = h->alloc<double>(s);
        l.cw.cE = h->alloc<double>(s);
        l.cw.cN = h->alloc<double>(s);
        l.cw.cNE = h->alloc<double>(s);
        l.cw.dinv = h->alloc<double>(s);
        l.cw.tab = h->alloc<double>(8 * (size_t)(l.g.n + 1) * l.cap);
      }
    } else {
      for (int q = 0; q < 8; ++q) l.c3.a[q] = h->alloc<double>(s);
      l.c3.dinv = h->alloc<double>(s);
      l.c3.tab = h->alloc<double>(15 * (size_t)(l.g.n + 1) * l.cap);
      for (int q = 0; q < 8; ++q) l.b3.a[q] = h->alloc<double>(s);
      l.cw3 = l.c3;
      if (h->literal()) {
        for (int q = 0; q < 8; ++q) l.cw3.a[q] = h->alloc<double>(s);
        l.cw3.dinv = h->alloc<double>(s);
        l.cw3.tab = h->alloc<double>(15 * (size_t)(l.g.n + 1) * l.cap);
      }
    }
    if (h->mixed()) {
      // single-precision V-cycle arrays: FP32, or bfloat16 storage (2 bytes) behind float*
      auto single = [&]() {
        return h->bf16() ? reinterpret_cast<float*>(h->alloc<uint16_t>(s)) : h->alloc<float>(s);
      };
      l.ct.tab = h->alloc<float>((size_t)(dim == 2 ? 8 : 15) * (l.g.n + 1) * l.cap);
      l.ct.tablo = h->alloc<float>((size_t)(dim == 2 ? 8 : 15) * (l.g.n + 1) * l.cap);
      l.ct.cst = h->alloc<float>(kCst * (size_t)l.cap);
      l.x32 = single();
      l.xt32 = single();
      l.f32 = single();
      l.r32 = single();
      l.uhi = h->alloc<float>(s);
      l.ulo = h->alloc<float>(s);
      if (!h->dry && tma_sweep_applies(l.g) && !(h->prob.flags & FMG_FLAG_NO_TMA)) {
        const bool bf = h->bf16();
        l.tma = encode_level_map(l.g, l.cap, l.x32, bf, true, &l.tm_x[0]) &&
                encode_level_map(l.g, l.cap, l.xt32, bf, true, &l.tm_x[1]) &&
                encode_level_map(l.g, l.cap, l.f32, bf, false, &l.tm_f);
        l.tm_base[0] = l.x32;
        l.tm_base[1] = l.xt32;
      }
    }
    l.x = h->alloc<double>(s);
    l.xt = h->alloc<double>(s);
    l.f = h->alloc<double>(s);
    l.r = h->alloc<double>(s);
    l.u = h->alloc<double>(s);
    l.y = h->alloc<double>(s);
    l.z = h->alloc<double>(s);
    if (k >= 2) {
      const int r = 1 << (k - 1);
      std::vector<double> pw(4 * (r + 1));  // (x/r)^m, m = 0..3, of the T3 sums
      t3_power_table(r, pw.data());
      l.pw = h->alloc<double>(pw.size());
      if (!h->dry) cudaMemcpyAsync(l.pw, pw.data(), pw.size() * sizeof(double), cudaMemcpyHostToDevice,
                h->stream);
      if (dim == 2) {
        double map[2 * 10 * 25];
        t3_map2d(r, map);
        l.t3map = h->alloc<double>(2 * 10 * 25);
        if (!h->dry) cudaMemcpyAsync(l.t3map, map, sizeof(map), cudaMemcpyHostToDevice,
                  h->stream);
      } else {
        std::vector<double> map(20 * 15 * 20);
        t3_map3d(r, map.data());
        l.t3map = h->alloc<double>(map.size());
        if (!h->dry) cudaMemcpyAsync(l.t3map, map.data(), map.size() * sizeof(double), cudaMemcpyHostToDevice,
                  h->stream);
      }
    }
  }
}

void build_coarse(fmg_eig_handle* h) {
  const int n1 = h->prob.coarse_cells;
  const int m = n1 - 1;
  const int dim = h->prob.dim;
  const int nb = h->nb;
  const double H = h->prob.box_len / n1;
  std::vector<int> tri, adj;
  if (dim == 2) {
    h->nh = m * m;
    h->nvert = 3;
    h->ntri = 2 * n1 * n1;
    h->maxadj = 6;
    h->tri_vol = H * H / 2.0;
    tri.resize(h->ntri * 3);
    auto id = [&](int i, int j) { return (i < 1 || j < 1 || i >= n1 || j >= n1) ? -1 : (i - 1) + (j - 1) * m; };
    for (int J = 0; J < n1; ++J)
      for (int I = 0; I < n1; ++I) {
        const int cell = I + n1 * J;
        const int t0[3] = {id(I, J), id(I + 1, J), id(I + 1, J + 1)};
        const int t1[3] = {id(I, J), id(I + 1, J + 1), id(I, J + 1)};
        for (int v = 0; v < 3; ++v) {
          tri[(2 * cell) * 3 + v] = t0[v];
          tri[(2 * cell + 1) * 3 + v] = t1[v];
        }
      }
  } else {
    h->nh = m * m * m;
    h->nvert = 4;
    h->ntri = 6 * n1 * n1 * n1;
    h->maxadj = 24;
    h->tri_vol = H * H * H / 6.0;
    tri.resize(h->ntri * 4);
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    auto id = [&](int i, int j, int l) {
      return (i < 1 || j < 1 || l < 1 || i >= n1 || j >= n1 || l >= n1)
                 ? -1 : (i - 1) + (j - 1) * m + (l - 1) * m * m;
    };
    for (int L = 0; L < n1; ++L)
      for (int J = 0; J < n1; ++J)
        for (int I = 0; I < n1; ++I) {
          const int cell = I + n1 * (J + n1 * L);
          for (int sp = 0; sp < 6; ++sp) {
            int v[3] = {I, J, L};
            int* out = &tri[(6 * cell + sp) * 4];
            out[0] = id(v[0], v[1], v[2]);
            v[perm[sp][0]]++;
            out[1] = id(v[0], v[1], v[2]);
            v[perm[sp][1]]++;
            out[2] = id(v[0], v[1], v[2]);
            out[3] = id(I + 1, J + 1, L + 1);
          }
        }
  }
  const int nv = h->nvert;
  adj.assign(h->nh * h->maxadj, -1);
  std::vector<int> fill(h->nh, 0);
  for (int t = 0; t < h->ntri; ++t)
    for (int v = 0; v < nv; ++v) {
      const int a = tri[t * nv + v];
      if (a >= 0) adj[a * h->maxadj + fill[a]++] = (t << 3) | v;
    }
  // gather lists of the dense solve's G(c) assembly: for each entry (a, b) with a simplex
  // around a that has b as a vertex, the simplex-local indices in a's adjacency order
  std::vector<int> gent, gstart{0}, gidx;
  {
    const int L = nv + 1;
    for (int a = 0; a < h->nh; ++a)
      for (int b = 0; b < h->nh; ++b) {
        const size_t before = gidx.size();
        for (int k = 0; k < h->maxadj; ++k) {
          const int code = adj[a * h->maxadj + k];
          if (code < 0) break;
          const int t = code >> 3, la = code & 7;
          for (int lb = 0; lb < nv; ++lb)
            if (tri[t * nv + lb] == b) gidx.push_back(t * L * L + la * L + lb);
        }
        if (gidx.size() > before) {
          gent.push_back(a * h->nh + b);
          gstart.push_back((int)gidx.size());
        }
      }
  }
  h->npat = (int)gent.size();
  h->tri = h->alloc<int>(tri.size());
  h->adj = h->alloc<int>(adj.size());
  h->gent = h->alloc<int>(gent.size());
  h->gstart = h->alloc<int>(gstart.size());
  h->gidx = h->alloc<int>(gidx.size());
  if (!h->dry) {
    cudaMemcpyAsync(h->tri, tri.data(), tri.size() * sizeof(int), cudaMemcpyHostToDevice,
                    h->stream);
    cudaMemcpyAsync(h->adj, adj.data(), adj.size() * sizeof(int), cudaMemcpyHostToDevice,
                    h->stream);
    cudaMemcpyAsync(h->gent, gent.data(), gent.size() * sizeof(int), cudaMemcpyHostToDevice,
                    h->stream);
    cudaMemcpyAsync(h->gstart, gstart.data(), gstart.size() * sizeof(int),
                    cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->gidx, gidx.data(), gidx.size() * sizeof(int), cudaMemcpyHostToDevice,
                    h->stream);
  }
  const size_t nn = (size_t)h->nh * h->nh;
  h->L1 = h->alloc<double>(nn * nb);
  h->L1A = h->literal() ? h->alloc<double>(nn * nb) : h->L1;
  h->M1 = h->alloc<double>(nn * nb);
  h->L1inv = h->alloc<double>(nn * nb);
  h->lam = h->alloc<double>(nb);
  h->c = h->alloc<double>((size_t)(h->nh + 1) * nb);
  h->cstart = h->alloc<double>((size_t)(h->nh + 1) * nb);
  h->auu = h->alloc<double>(nb);
  h->buu = h->alloc<double>(nb);
  h->scal = h->alloc<double>(3 * (size_t)nb + 8);
  h->partials = h->alloc<double>((size_t)kReduceBlocks * nb);
  if (h->prob.smoother == FMG_SMOOTH_CG) h->cg = h->alloc<double>(3 * (size_t)nb);
  h->partials2 = h->alloc<double>((size_t)kReduceBlocks * nb);
  const int nt3 = dim == 2 ? 10 : 20;
  h->t3 = h->alloc<double>((size_t)h->ntri * nt3 * nb);
  size_t tp = 1;
  for (int k = 2; k <= h->levels(); ++k) {
    const Grid& g = h->L(k).g;
    tp = std::max(tp, (dim == 2 ? t3_partials2d(g, n1) : t3_partials3d(g, n1)) * h->cnt[k]);
  }
  h->t3_partials = h->alloc<double>(tp);
  h->gAd = h->alloc<double>((size_t)h->nh * nb);
  h->gMd = h->alloc<double>((size_t)h->nh * nb);
  h->t1d = h->alloc<double>((size_t)h->nh * nb);
  h->B1d = h->alloc<double>(nn * nb);
  h->t0 = h->alloc<double>(nb);
  h->kscratch = h->alloc<double>(3 * (size_t)(h->nh + 1) * (h->nh + 1) + h->nh + 1);
  h->lam_levels = h->alloc<double>((size_t)FMG_MAX_LEVELS * nb);
  h->iters = h->alloc<int>((size_t)FMG_MAX_LEVELS * nb);
  h->status = h->alloc<int>((size_t)FMG_MAX_LEVELS * nb);
  h->wait_fail = h->alloc<int>(nb);
  size_t tot = 0;
  h->uoff.resize(nb);
  for (int b = 0; b < nb; ++b) {
    h->uoff[b] = tot;
    tot += h->L(h->probs[b].levels).g.interior();
  }
  h->uout = h->alloc<double>(tot);
  std::vector<int> inv(nb);
  for (int b = 0; b < nb; ++b) inv[h->order[b]] = b;
  h->inv_order = h->alloc<int>(nb);
  if (!h->dry) cudaMemcpyAsync(h->inv_order, inv.data(), sizeof(int) * nb, cudaMemcpyHostToDevice,
                  h->stream);
  h->dense_smem = dense_smem_bytes(h->nh + 1, h->ntri, h->nvert, 1);
}

// (Every build-time upload above goes through the handle's stream from pageable host memory:
// the call returns once the source is staged, and the allocations it targets are ordered on
// the same stream.)

// ---- enqueue helpers (all work in stream order on s) ---------------------------------------
void prof_begin(fmg_eig_handle* h, int id, int level, cudaStream_t s) {
  if (level == h->levels() && h->prof_armed[id])
    cudaEventRecordWithFlags(h->prof[id][0], s, cudaEventRecordExternal);
}
void prof_end(fmg_eig_handle* h, int id, int level, cudaStream_t s) {
  if (level == h->levels() && h->prof_armed[id]) {
    cudaEventRecordWithFlags(h->prof[id][1], s, cudaEventRecordExternal);
    h->prof_armed[id] = false;
  }
}

// s waits for the side streams' work so far: [first, first + count) of side[]
void join_sides(fmg_eig_handle* h, cudaStream_t s, int first, int count) {
  for (int i = first; i < first + count; ++i) {
    cudaEventRecord(h->ev_join[i], h->side[i]);
    cudaStreamWaitEvent(s, h->ev_join[i], 0);
  }
}
void fork_sides(fmg_eig_handle* h, cudaStream_t s, int first, int count) {
  cudaEventRecord(h->ev_fork, s);
  for (int i = first; i < first + count; ++i) cudaStreamWaitEvent(h->side[i], h->ev_fork, 0);
}

// The operators of level k must be ready on s from here on (setup forked in enqueue_setup).
void need_level(fmg_eig_handle* h, int k, cudaStream_t s) {
  if (!h->level_pending[k]) return;
  cudaStreamWaitEvent(s, h->ev_level[k], 0);
  h->level_pending[k] = false;
}

// Operators of every level for every instance that has the level, and the level-1 inverse.
// With `overlap`, levels >= 2 are built on a side stream while the coarse solve runs, and
// each stage joins the levels it needs (need_level).
void enqueue_setup(fmg_eig_handle* h, cudaStream_t s, bool overlap = false) {
  h->activate(h->nb);
  if (overlap && h->levels() >= 2) fork_sides(h, s, 2, 1);
  for (int k = 1; k <= h->levels(); ++k) {
    Level& l = h->L(k);
    const cudaStream_t sk = overlap && k >= 2 ? h->side[2] : s;
    const cudaStream_t s_saved = s;
    s = sk;
    prof_begin(h, kProfCoef, k, s);
    lv_coef(l, h->dparams, s);
    if (h->literal()) lv_coef(l, h->dparams_full, s, true);
    prof_end(h, kProfCoef, k, s);
    if (h->mixed()) tables_f32(l.g, l.c, l.c3, h->dparams, l.ct, s);
    if (sk != s_saved) {
      cudaEventRecord(h->ev_level[k], sk);
      h->level_pending[k] = true;
    }
    s = s_saved;
  }
  lv_dense_level1(h->L(1), h->L1, h->M1, s, true);
  if (h->literal()) lv_dense_level1(h->L(1), h->L1A, h->M1, s, false);
  dense_spd_inverse(h->L1A, h->L1inv, h->nh, h->L(1).g.nb, s);
}

DenseProblem dense_base(fmg_eig_handle* h) {
  DenseProblem d{};
  d.nh = h->nh;
  d.ntri = h->ntri;
  d.nvert = h->nvert;
  d.tri = h->tri;
  d.adj = h->adj;
  d.maxadj = h->maxadj;
  d.npat = h->npat;
  d.gent = h->gent;
  d.gstart = h->gstart;
  d.gidx = h->gidx;
  d.quart_off = h->tri_vol * 2.0 * factorial(h->prob.dim) / factorial(h->prob.dim + 4);
  d.tri_vol = h->tri_vol;
  d.L1 = h->L1;
  d.M1 = h->M1;
  d.nt3 = h->prob.dim == 2 ? 10 : 20;
  d.params = h->dparams;
  d.tol = h->prob.scf_tol;
  d.max_iter = h->prob.scf_max_iter;
  d.c_out = h->c;
  d.lam_out = h->lam;
  return d;
}

// Algorithm 3.2 step 1 into L(1).u and h->lam for the active instances
void enqueue_coarse(fmg_eig_handle* h, cudaStream_t s) {
  Level& l1 = h->L(1);
  lv_start(l1, h->cstart, h->nh + 1, s);
  DenseProblem d = dense_base(h);
  d.aug = 0;
  d.c_init = h->cstart;
  d.iters_out = h->iters;
  d.status_out = h->status;
  dense_scf(d, l1.g.nb, s);
  scatter_level1(l1.g, h->c, h->nh + 1, l1.u, s);
}

// Chebyshev semi-iteration of degree nu on the interval [kChebLow, kChebHigh] of the spectrum
// of D^{-1} L: the upper end is Gershgorin's bound for these operators (stiffness rows sum
// to zero, the potential mass has the P1 mass pattern, so |off-diagonal| row sums of
// D^{-1} L are at most 1); the smoother damps the spectrum above the lower end.  Three-term
// recurrence of Chebyshev acceleration: theta, delta the interval's centre and half-width,
// sigma = theta / delta, rho_0 = 1 / sigma, rho_k = 1 / (2 sigma - rho_{k-1});
// step 0: d = D^{-1} r / theta; step k: d = rho_k rho_{k-1} d + (2 rho_k / delta) D^{-1} r.
constexpr double kChebLow = 0.3, kChebHigh = 2.0;

void cheb_coefficients(int nu, std::vector<double>& alpha, std::vector<double>& beta) {
  const double theta = 0.5 * (kChebHigh + kChebLow), delta = 0.5 * (kChebHigh - kChebLow);
  const double sigma = theta / delta;
  alpha.assign(nu, 0.0);
  beta.assign(nu, 0.0);
  if (nu < 1) return;
  beta[0] = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int k = 1; k < nu; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    alpha[k] = rn * rho;
    beta[k] = 2.0 * rn / delta;
    rho = rn;
  }
}

// nu smoothing steps on level l (x, f in l.x, l.f; the result ends in l.x)
void enqueue_smooth(fmg_eig_handle* h, Level& l, int j, int nu, bool& zero, cudaStream_t s) {
  if (h->prob.smoother == FMG_SMOOTH_CG) {
    // nu CG steps on L x = f from x (Section 4): r in l.r, direction p in l.z, q = L p in l.y;
    // per-instance scalars r.r (two slots, old / new) and p.q in h->cg
    if (nu <= 0) return;
    const size_t st = l.g.stride, n = st * l.g.nb;
    if (zero) {
      cudaMemsetAsync(l.x, 0, n * sizeof(double), s);
      cudaMemcpyAsync(l.r, l.f, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
      lv_residual(l, l.f, l.x, l.r, s);
    }
    zero = false;
    cudaMemcpyAsync(l.z, l.r, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    double* rr = h->cg;
    double* rr_new = h->cg + h->nb;
    double* pq = h->cg + 2 * h->nb;
    dot(l.r, l.r, st, h->partials, rr, s, l.g.nb, st);
    for (int it = 0; it < nu; ++it) {
      lv_apply(l, l.z, l.y, s);
      dot(l.z, l.y, st, h->partials, pq, s, l.g.nb, st);
      cg_update(n, st, rr, pq, l.z, l.y, l.x, l.r, s);
      dot(l.r, l.r, st, h->partials, rr_new, s, l.g.nb, st);
      cg_direction(n, st, rr_new, rr, l.r, l.z, s);
      std::swap(rr, rr_new);
    }
    return;
  }
  if (h->prob.smoother == FMG_SMOOTH_CHEBYSHEV) {
    std::vector<double> al, be;
    cheb_coefficients(nu, al, be);
    for (int it = 0; it < nu; ++it) {
      const bool prof = !zero;
      if (prof) prof_begin(h, kProfJacobi, j, s);
      lv_cheb(l, l.f, l.x, l.z, l.xt, al[it], be[it], it == 0, zero, s);
      if (prof) prof_end(h, kProfJacobi, j, s);
      std::swap(l.x, l.xt);
      zero = false;
    }
    return;
  }
  for (int it = 0; it < nu; ++it) {
    const bool prof = !zero;
    if (prof) prof_begin(h, kProfJacobi, j, s);
    lv_jacobi(l, l.f, l.x, l.xt, zero, s);
    if (prof) prof_end(h, kProfJacobi, j, s);
    std::swap(l.x, l.xt);
    zero = false;
  }
}

// The whole V-cycle from level j in one kernel (vcycle_small.cu) when level j is small: 2D,
// damped Jacobi, at most 32 cells per side.  The result lands in L(j).x; the levels below
// keep their vectors in shared memory.
bool enqueue_vcycle_fused(fmg_eig_handle* h, int j, bool x_zero, cudaStream_t s) {
  const fmg_eig_problem& p = h->prob;
  if (p.dim != 2 || p.smoother != FMG_SMOOTH_JACOBI || (p.flags & FMG_FLAG_SEPARATE_VCYCLE))
    return false;
  if (j < 2 || j > kSmallMaxLevels || h->L(j).g.n > kSmallMaxCells) return false;
  SmallVcycle v{};
  v.levels = j;
  v.nu_pre = p.nu_pre;
  v.nu_post = p.nu_post;
  v.x_zero = x_zero ? 1 : 0;
  for (int k = 1; k <= j; ++k) {
    const Level& l = h->L(k);
    v.lv[k - 1] = SmallLevel2D{l.g.n, l.g.pitch, l.g.stride, l.c};
  }
  v.Linv = h->L1inv;
  v.f = h->L(j).f;
  v.x = h->L(j).x;
  return vcycle_small(v, h->L(j).g.nb, s) == cudaSuccess;
}

// One V-cycle on level j for L_j x = f (x, f in L(j).x, L(j).f).
void enqueue_vcycle(fmg_eig_handle* h, int j, bool x_zero, cudaStream_t s) {
  Level& l = h->L(j);
  if (j == 1) {
    coarse_matvec(l.g, h->L1inv, l.f, l.x, s);
    return;
  }
  if (enqueue_vcycle_fused(h, j, x_zero, s)) return;
  const fmg_eig_problem& p = h->prob;
  bool zero = x_zero;
  prof_begin(h, kProfVcycle, j, s);
  enqueue_smooth(h, l, j, p.nu_pre, zero, s);
  if (zero) cudaMemsetAsync(l.x, 0, l.g.stride * l.g.nb * sizeof(double), s);
  Level& lc = h->L(j - 1);
  prof_begin(h, kProfResidual, j, s);
  lv_residual(l, l.f, l.x, l.r, s);
  prof_end(h, kProfResidual, j, s);
  prof_begin(h, kProfRestrict, j, s);
  lv_restrict(l, lc, l.r, lc.f, s);
  prof_end(h, kProfRestrict, j, s);
  enqueue_vcycle(h, j - 1, true, s);
  prof_begin(h, kProfProlong, j, s);
  lv_prolong(l, lc, lc.x, l.x, true, nullptr, nullptr, 0, s);
  prof_end(h, kProfProlong, j, s);
  bool post_zero = false;
  enqueue_smooth(h, l, j, p.nu_post, post_zero, s);
  prof_end(h, kProfVcycle, j, s);
}

// Single-precision sweep (mode 0 residual into r32, 1 Jacobi, 2 Jacobi from zero, both into
// xt32) of level l: TMA-fed on the large 2D levels, register-blocked otherwise.
void lv_sweep32(fmg_eig_handle* h, Level& l, int mode, cudaStream_t s) {
  const bool bf = h->bf16();
  if (l.tma) {
    const TMAMap& mx = l.x32 == l.tm_base[0] ? l.tm_x[0] : l.tm_x[1];
    sweep32_tma(l.g, l.ct, mx, l.tm_f, mode == 0 ? l.r32 : l.xt32, mode, h->wait_fail,
                (h->prob.flags & FMG_FLAG_EXPIRE_WAITS) != 0, s, bf);
  } else if (mode == 0) {
    residual32(l.g, l.ct, l.f32, l.x32, l.r32, s, bf);
  } else {
    jacobi32(l.g, l.ct, l.f32, l.x32, l.xt32, mode == 2, s, bf);
  }
}

// One FP32 V-cycle on level j for L_j e = r (e, r in L(j).x32, L(j).f32), e starting at 0.
void enqueue_vcycle32(fmg_eig_handle* h, int j, cudaStream_t s) {
  Level& l = h->L(j);
  const bool bf = h->bf16();
  if (j == 1) {
    coarse32(l.g, h->L1inv, l.f32, l.x32, s, bf);
    return;
  }
  const fmg_eig_problem& p = h->prob;
  if (!l.tma && !(p.flags & FMG_FLAG_SEPARATE_VCYCLE) &&
      vcycle32_mid_applies(l.g, p.nu_pre, p.nu_post)) {
    // both legs of the level in one kernel each (vcycle32_mid.cu), same results
    Level& lc = h->L(j - 1);
    vcycle32_down(l.g, l.ct, lc.g, l.f32, l.x32, lc.f32, p.nu_pre, s, bf);
    enqueue_vcycle32(h, j - 1, s);
    vcycle32_up(l.g, l.ct, lc.g, l.f32, l.x32, l.xt32, lc.x32, p.nu_post, s, bf);
    std::swap(l.x32, l.xt32);
    return;
  }
  bool zero = true;
  for (int it = 0; it < p.nu_pre; ++it) {
    // the profiled sweep is the first one that reads x (the zero-start sweep reads only f)
    const bool prof = !zero;
    if (prof) prof_begin(h, kProfJacobi, j, s);
    lv_sweep32(h, l, zero ? 2 : 1, s);
    if (prof) prof_end(h, kProfJacobi, j, s);
    std::swap(l.x32, l.xt32);
    zero = false;
  }
  if (zero) cudaMemsetAsync(l.x32, 0, l.g.stride * l.g.nb * mixed_elem_bytes(bf), s);
  Level& lc = h->L(j - 1);
  prof_begin(h, kProfResidual, j, s);
  lv_sweep32(h, l, 0, s);
  prof_end(h, kProfResidual, j, s);
  prof_begin(h, kProfRestrict, j, s);
  restrict32(l.g, lc.g, l.r32, lc.f32, s, bf);
  prof_end(h, kProfRestrict, j, s);
  enqueue_vcycle32(h, j - 1, s);
  prof_begin(h, kProfProlong, j, s);
  prolong32_add(l.g, lc.g, lc.x32, l.x32, s, bf);
  prof_end(h, kProfProlong, j, s);
  for (int it = 0; it < p.nu_post; ++it) {
    lv_sweep32(h, l, 1, s);
    std::swap(l.x32, l.xt32);
  }
}

// The m multigrid iterations of Algorithm 3.1 step 1 on level k.  In the mixed modes an FMG
// stage whose level is large enough for bandwidth to matter (the levels of the TMA-fed
// sweeps: n >= 512 in 2D, >= 128 in 3D) runs FP64 defect correction around single-precision
// V-cycles; smaller stages, where the V-cycle is bound by latency rather than bandwidth, run
// the FP64 V-cycles (in_fmg = false, the component call, always takes the mixed path).  The
// early stages then match the FP64 solve exactly: with a strong nonlinearity (3D, zeta ~
// 150-200) single-precision rounding entering there grew to |d lambda| ~1e-8 at the end.
void enqueue_multigrid(fmg_eig_handle* h, int k, cudaStream_t s, bool in_fmg = true) {
  if (h->mixed() && (!in_fmg || tma_sweep_applies(h->L(k).g))) {
    // FP64 defect correction around single-precision V-cycles
    Level& l = h->L(k);
    for (int it = 0; it < h->prob.vcycles; ++it) {
      prof_begin(h, kProfVcycle, k, s);
      residual_mixed(l.g, l.c, l.c3, l.f, l.x, l.f32, s, h->bf16());
      enqueue_vcycle32(h, k, s);
      add_f32(l.x32, l.x, l.g.stride * l.g.nb, s, h->bf16());
      prof_end(h, kProfVcycle, k, s);
    }
    return;
  }
  for (int it = 0; it < h->prob.vcycles; ++it) enqueue_vcycle(h, k, false, s);
}

// Fine pass of the augmented problem on level k for u~ (Algorithm 3.1 step 2): the linear
// blocks g_A = P^T..P^T L u~, g_M = P^T..P^T M u~, u~^T L u~, u~^T M u~, and the moments
// T0, T1 (restricted cubic load), T2 (coarsened density stencil), T3 (per coarse triangle),
// gathered into the dense level-1 arrays of the handle.
void enqueue_augment(fmg_eig_handle* h, int k, const double* ut, cudaStream_t s) {
  Level& l = h->L(k);
  const int nb = l.g.nb;
  const size_t st = l.g.stride;
  // FP64 mode: N(u~) and B(u~) run alone first.  Every kernel of the pass is bound by the
  // FP64 pipe, so running the T3 sums and the operator applies beside it gains nothing; the
  // branches below then overlap the short restriction / coarsening chains.  The mixed modes
  // compute it in double-float on the FP32 pipes, beside the FP64 T3 sums and applies.
  if (!h->mixed()) {
    prof_begin(h, kProfMoments, k, s);
    lv_nload_density(l, ut, l.r, s);
    prof_end(h, kProfMoments, k, s);
  }
  // mixed modes: the double-float split of u~, read by N(u~) / B(u~) and by the mass apply
  const SplitVec us = h->mixed() ? lv_split(l, ut, s) : SplitVec{};
  fork_sides(h, s, 0, 2);
  // branch 1 (side 0): N(u~) and B(u~) (mixed modes), T0, and the restriction / coarsening
  // chains of both
  {
    const cudaStream_t b1 = h->side[0];
    if (h->mixed()) {
      prof_begin(h, kProfMoments, k, b1);
      lv_nload_density_df(l, us, l.r, b1);
      prof_end(h, kProfMoments, k, b1);
    }
    dot(ut, l.r, st, h->partials2, h->t0, b1, nb, st);
    for (int j = k; j >= 2; --j) {
      lv_restrict(h->L(j), h->L(j - 1), h->L(j).r, h->L(j - 1).r, b1);
      lv_coarsen_density(h->L(j), h->L(j - 1), b1, h->mixed());
    }
  }
  // branch 2 (side 1): T3 per coarse simplex
  {
    const cudaStream_t b2 = h->side[1];
    prof_begin(h, kProfT3, k, b2);
    lv_t3(l, h->prob.coarse_cells, ut, h->t3_partials, h->t3, b2);
    prof_end(h, kProfT3, k, b2);
  }
  // main branch: (A + W) u~, M u~, their dots and restriction chains.  The mixed modes form
  // M u~ in double-float on the FP32 pipes (positive weights: ~2^-47 of the result); the
  // operator apply stays FP64 (its stencil cancels to O(h^2) of its terms).
  lv_apply_full(l, ut, l.y, s);
  if (h->mixed()) lv_mass_df(l, us, l.z, s);
  else lv_mass(l, ut, l.z, s);
  dot(ut, l.y, st, h->partials, h->auu, s, nb, st);
  dot(ut, l.z, st, h->partials, h->buu, s, nb, st);
  for (int j = k; j >= 2; --j)  // both chains in one launch per level
    lv_restrict(h->L(j), h->L(j - 1), h->L(j).y, h->L(j - 1).y, s, h->L(j).z, h->L(j - 1).z);
  join_sides(h, s, 0, 2);
  Level& l1 = h->L(1);
  lv_gather_level1(l1, h->gAd, h->gMd, h->t1d, h->B1d, s, h->mixed());
}

DenseProblem dense_augmented(fmg_eig_handle* h) {
  DenseProblem d = dense_base(h);
  d.aug = 1;
  d.gA = h->gAd;
  d.gM = h->gMd;
  d.t1 = h->t1d;
  d.B1 = h->B1d;
  d.t3 = h->t3;
  d.auu = h->auu;
  d.buu = h->buu;
  d.t0 = h->t0;
  return d;
}

// One correction step (Algorithm 3.1) on level k for the active instances:
// (h->lam, L(k).u) -> (h->lam, L(k).u); u~ stays in L(k).x.
void enqueue_correction(fmg_eig_handle* h, int k, cudaStream_t s) {
  Level& l = h->L(k);
  const int nb = l.g.nb;
  // step 1: auxiliary problem, m V-cycles from u
  prof_begin(h, kProfRhs, k, s);
  if (h->mixed() && (h->prob.flags & FMG_FLAG_FP32_RHS))
    lv_rhs_f32(l, h->lam, h->dparams, l.u, l.f, s);
  else if (h->mixed())
    lv_rhs_df(l, h->lam, h->dparams, l.u, l.f, s);
  else lv_rhs(l, h->lam, h->dparams, l.u, l.f, s);
  if (h->literal()) lv_sub_wmass(l, l.u, l.f, s);
  prof_end(h, kProfRhs, k, s);
  cudaMemcpyAsync(l.x, l.u, l.g.stride * nb * sizeof(double), cudaMemcpyDeviceToDevice, s);
  enqueue_multigrid(h, k, s);
  const double* ut = l.x;
  // step 2: augmented space V_H + span{u~}
  enqueue_augment(h, k, ut, s);
  DenseProblem d = dense_augmented(h);
  d.c_init = nullptr;
  d.iters_out = h->iters + (size_t)(k - 1) * h->nb;
  d.status_out = h->status + (size_t)(k - 1) * h->nb;
  prof_begin(h, kProfDense, k, s);
  dense_scf(d, nb, s);
  prof_end(h, kProfDense, k, s);
  // u = P_{k<-1} c_H + c_u u~
  scatter_level1(h->L(1).g, h->c, h->nh + 1, h->L(1).y, s);
  for (int j = 2; j < k; ++j)
    lv_prolong(h->L(j), h->L(j - 1), h->L(j - 1).y, h->L(j).y, false, nullptr, nullptr, 0, s);
  lv_prolong(l, h->L(k - 1), h->L(k - 1).y, l.u, false, ut, h->c + h->nh, h->nh + 1, s);
}

void enqueue_fmg(fmg_eig_handle* h, cudaStream_t s, const StageHook* after_stage) {
  cudaMemsetAsync(h->wait_fail, 0, sizeof(int) * h->nb, s);  // no bounded wait gave up yet
  enqueue_setup(h, s, true);
  h->activate(h->nb);
  enqueue_coarse(h, s);
  cudaMemcpyAsync(h->lam_levels, h->lam, sizeof(double) * h->nb, cudaMemcpyDeviceToDevice, s);
  if (after_stage && h->cnt[1] > h->cnt[2]) (*after_stage)(1, h->cnt[2], h->cnt[1] - h->cnt[2]);
  for (int k = 2; k <= h->levels(); ++k) {
    need_level(h, k, s);
    h->activate(h->cnt[k]);
    lv_prolong(h->L(k), h->L(k - 1), h->L(k - 1).u, h->L(k).u, false, nullptr, nullptr, 0, s);
    for (int it = 0; it < h->prob.corrections; ++it) enqueue_correction(h, k, s);
    cudaMemcpyAsync(h->lam_levels + (size_t)(k - 1) * h->nb, h->lam, sizeof(double) * h->cnt[k],
                    cudaMemcpyDeviceToDevice, s);
    if (after_stage && h->cnt[k] > h->cnt[k + 1])
      (*after_stage)(k, h->cnt[k + 1], h->cnt[k] - h->cnt[k + 1]);
  }
  h->activate(1);
}

// u of every instance, unpacked from its finest level into h->uout (per level group).
void enqueue_outputs(fmg_eig_handle* h, cudaStream_t s) {
  for (int k = 1; k <= h->levels(); ++k) {
    const int first = h->cnt[k + 1], count = h->cnt[k] - h->cnt[k + 1];
    if (count <= 0) continue;
    Level v = view(h->L(k), first, count);
    unpack_interior(v.g, v.u, h->uout + h->uoff[first], s);
  }
}

// b(u,u), a(u,u) + (Wu,u) and int u^4 of every instance's final u into h->scal (3 x nb).
void enqueue_checks(fmg_eig_handle* h, cudaStream_t s) {
  double* sa = h->scal;
  double* sb = h->scal + h->nb;
  double* sn = h->scal + 2 * h->nb;
  for (int k = 1; k <= h->levels(); ++k) {
    const int first = h->cnt[k + 1], count = h->cnt[k] - h->cnt[k + 1];
    if (count <= 0) continue;
    Level v = view(h->L(k), first, count);
    const size_t st = v.g.stride;
    lv_apply_full(v, v.u, v.y, s);
    lv_mass(v, v.u, v.z, s);
    lv_nload(v, v.u, v.r, s);
    dot(v.u, v.y, st, h->partials, sa + first, s, count, st);
    dot(v.u, v.z, st, h->partials, sb + first, s, count, st);
    dot(v.u, v.r, st, h->partials, sn + first, s, count, st);
  }
}

cudaStream_t pick(fmg_eig_handle* h, void* stream) {
  return stream ? static_cast<cudaStream_t>(stream) : h->stream;
}

bool level_ok(const fmg_eig_handle* h, int k) { return h && k >= 1 && k <= h->prob.levels; }

// ---- autotuner: thread-block shape per level -----------------------------------------------
// The stencil kernels of a level compute every node with the same expression whatever the
// block shape, so the shape only changes the time.  For each level the tuner times a small
// mix of that level's launches (4 Jacobi sweeps, one cubic-load + density pass, one RHS) per
// candidate shape on the handle's own buffers, keeps the fastest, and remembers the choice
// per (dim, n, instances rounded up to a power of two, precision) for the process.
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune_cache;

void time_mix(fmg_eig_handle* h, Level& l, int k, cudaStream_t s) {
  for (int q = 0; q < 4; ++q) {
    if (h->mixed() && k >= 2)
      jacobi32(l.g, l.ct, l.f32, l.x32, l.xt32, false, s, h->bf16());
    else
      lv_jacobi(l, l.f, l.x, l.xt, false, s);
  }
  if (h->mixed()) {
    lv_nload_density_df(l, lv_split(l, l.u, s), l.r, s);
    lv_rhs_df(l, h->lam, h->dparams, l.u, l.f, s);
  } else {
    lv_nload_density(l, l.u, l.r, s);
    lv_rhs(l, h->lam, h->dparams, l.u, l.f, s);
  }
}

int autotune(fmg_eig_handle* h) {
  if ((h->prob.flags & FMG_FLAG_NO_AUTOTUNE) || h->opt.tune == 0) return FMG_OK;
  static const int k2d[][2] = {{32, 8}, {32, 4}, {64, 4}, {32, 16}, {128, 2},
                               {64, 8}, {16, 16}, {16, 8}, {8, 8},  {8, 4}};
  static const int k3d[][2] = {{32, 8}, {32, 4}, {64, 2}, {32, 2}, {64, 4},
                               {16, 8}, {8, 8},  {16, 4}};
  cudaStream_t s = h->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FMG_ECUDA;
  }
  int rc = FMG_OK;
  for (int k = 1; k <= h->levels() && rc == FMG_OK; ++k) {
    Level& l = h->L(k);
    l.g.nb = l.cap;
    int nbq = 1;
    while (nbq < l.cap) nbq <<= 1;
    const auto key = std::make_tuple(l.g.dim, l.g.n, nbq, h->prob.precision);
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        l.g.bx = it->second.first;
        l.g.by = it->second.second;
        continue;
      }
    }
    if (h->opt.tune < 2) continue;  // cache only: keep the default shape
    const size_t nodes = l.g.interior() * (size_t)l.cap;
    const bool big = nodes >= ((size_t)1 << 20);
    const int ncand = l.g.dim == 2 ? (big ? 4 : 10) : (big ? 4 : 8);
    const int reps = big ? 1 : 5;
    float best = 1e30f;
    int bx = 32, by = 8;
    for (int ci = 0; ci < ncand; ++ci) {
      l.g.bx = l.g.dim == 2 ? k2d[ci][0] : k3d[ci][0];
      l.g.by = l.g.dim == 2 ? k2d[ci][1] : k3d[ci][1];
      time_mix(h, l, k, s);  // warm-up
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) time_mix(h, l, k, s);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        rc = FMG_ECUDA;
        break;
      }
      if (ms < best) {
        best = ms;
        bx = l.g.bx;
        by = l.g.by;
      }
    }
    l.g.bx = bx;
    l.g.by = by;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {bx, by};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->activate(1);
  return rc;
}

// Validation, the sorted instance order and the per-level counts of a new handle.
int init_instances(fmg_eig_handle* h, const fmg_eig_problem* probs, int count) {
  for (int i = 0; i < count; ++i) {
    const int v = validate(&probs[i]);
    if (v != FMG_OK) return v;
    if (shared_key(probs[i]) != shared_key(probs[0])) return FMG_EINVAL;
  }
  h->nb = count;
  h->order.resize(count);
  std::iota(h->order.begin(), h->order.end(), 0);
  std::stable_sort(h->order.begin(), h->order.end(),
                   [&](int a, int b) { return probs[a].levels > probs[b].levels; });
  for (int b = 0; b < count; ++b) h->probs.push_back(probs[h->order[b]]);
  h->prob = h->probs[0];
  h->cnt.assign(h->prob.levels + 2, 0);
  for (int k = 1; k <= h->prob.levels; ++k)
    for (const auto& p : h->probs) h->cnt[k] += p.levels >= k ? 1 : 0;
  if (h->prob.dim == 3)  // planes and instances share gridDim.z of the 3D launches
    for (int k = 1; k <= h->prob.levels; ++k)
      if ((size_t)((h->prob.coarse_cells << (k - 1)) + 1) * h->cnt[k] > 65535) return FMG_ENOTSUP;
  return FMG_OK;
}

size_t estimate_bytes(const fmg_eig_problem* probs, int count) {
  if (!probs || count < 1) return 0;
  fmg_eig_handle h;
  h.dry = true;
  if (init_instances(&h, probs, count) != FMG_OK) return 0;
  build_levels(&h);
  build_coarse(&h);
  h.alloc<PotentialParams>(h.literal() ? 2 * count : count);
  return h.bytes;
}

int create_handle(const fmg_eig_problem* probs, int count, const CreateOptions& opt,
                  fmg_eig_handle** out) {
  if (!out || !probs || count < 1) return FMG_EINVAL;
  *out = nullptr;
  fmg_eig_handle* h = new (std::nothrow) fmg_eig_handle();
  if (!h) return FMG_ENOMEM;
  h->opt = opt;
  const int vi = init_instances(h, probs, count);
  if (vi != FMG_OK) {
    delete h;
    return vi;
  }
  bool ok = cudaGetDevice(&h->dev) == cudaSuccess &&
            cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&h->ev0) == cudaSuccess && cudaEventCreate(&h->ev1) == cudaSuccess &&
            cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < 3; ++i)
    ok = cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking) == cudaSuccess &&
         (i == 2 || cudaEventCreateWithFlags(&h->ev_join[i], cudaEventDisableTiming) == cudaSuccess);
  for (int k = 0; ok && k <= h->prob.levels; ++k)
    ok = cudaEventCreateWithFlags(&h->ev_level[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    delete h;
    return FMG_ECUDA;
  }
  try {
    build_levels(h);
    build_coarse(h);
    h->nparams = h->literal() ? 2 * count : count;
    h->dparams = h->alloc<PotentialParams>(h->nparams);
    h->dparams_full = h->literal() ? h->dparams + count : h->dparams;
  } catch (const std::bad_alloc&) {
    delete h;
    return FMG_ENOMEM;
  }
  // pinned staging for the per-solve upload of a reusable handle; a one-shot handle (the
  // server's) uses pageable memory, whose release never waits for the device
  if (opt.async_alloc) {
    h->hparams = new (std::nothrow) PotentialParams[h->nparams];
    if (!h->hparams) {
      delete h;
      return FMG_ENOMEM;
    }
  } else if (cudaMallocHost(&h->hparams, sizeof(PotentialParams) * h->nparams) != cudaSuccess) {
    cudaGetLastError();
    h->hparams = nullptr;
    delete h;
    return FMG_ENOMEM;
  }
  fill_params(h);
  for (int i = 0; i < kProfCount; ++i)
    for (int j = 0; j < 2; ++j)
      if (cudaEventCreate(&h->prof[i][j]) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return FMG_ECUDA;
      }
  upload_params(h, h->stream);
  if (h->dense_smem > kDenseSmemLimit) {  // the small dense solve keeps everything in shared memory
    delete h;
    return FMG_ENOTSUP;
  }
  if (dense_prepare(h->dense_smem) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FMG_ECUDA;
  }
  // component entry points need the operators (the solve recomputes them itself), and the
  // tuner times launches on them
  const bool tune_runs = opt.tune == 2 && !(h->prob.flags & FMG_FLAG_NO_AUTOTUNE);
  if (opt.component_setup || tune_runs) {
    enqueue_setup(h, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return FMG_ECUDA;
    }
  }
  if (autotune(h) != FMG_OK) {
    delete h;
    return FMG_ECUDA;
  }
  h->activate(1);
  if (!opt.graph) {
    *out = h;
    return FMG_OK;
  }
  for (int i = 0; i < kProfCount; ++i) h->prof_armed[i] = true;
  // stage marks: one event per stage that finishes instances
  StageHook mark_hook = [h](int, int first, int count) {
    fmg_eig_handle::StageMark m{nullptr, first, count};
    if (cudaEventCreate(&m.ev) == cudaSuccess) {
      cudaMemcpyAsync(h->opt.stage_lam + first, h->lam + first, sizeof(double) * count,
                      cudaMemcpyDeviceToHost, h->stream);
      cudaEventRecordWithFlags(m.ev, h->stream, cudaEventRecordExternal);
    }
    h->marks.push_back(m);
  };
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_fmg(h, h->stream, opt.stage_lam ? &mark_hook : nullptr);
    e = cudaStreamEndCapture(h->stream, &h->graph);
  }
  for (const auto& m : h->marks)
    if (!m.ev && e == cudaSuccess) e = cudaErrorMemoryAllocation;
  for (int i = 0; i < kProfCount; ++i) h->prof_armed[i] = false;
  if (e == cudaSuccess) {
    size_t n = 0;
    e = cudaGraphGetNodes(h->graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(h->graph, nodes.data(), &n);
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      if (t == cudaGraphNodeTypeKernel) h->kernel_nodes++;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->exec, h->graph, 0);
  h->activate(1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return FMG_ECUDA;
  }
  *out = h;
  return FMG_OK;
}

// fmg_eig_inject_alloc_failure: the number of device allocations that still succeed before
// the chosen one fails (negative: none is chosen)
std::atomic<long long> g_alloc_fail_after{-1};

bool injected_alloc_failure() {
  long long v = g_alloc_fail_after.load();
  while (v >= 0)
    if (g_alloc_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

// Return code of sorted instance b (lb levels) from the per-level statuses of its small
// solves (st[level][instance]) and its bounded-wait word: a wait that gave up outranks an
// iteration cap that was hit.
int instance_code(const int* st, const int* wait_fail, int nb, int b, int lb) {
  if (wait_fail[b] != 0) return FMG_ETIMEOUT;
  for (int k = 1; k <= lb; ++k)
    if (st[(size_t)(k - 1) * nb + b] != 0) return FMG_ENOCONV;
  return FMG_OK;
}

// Launch the solve graph of every handle (each on its own stream), then collect the outputs
// of each in the callers' order.  out_index[h][b] is the caller's index of h's instance b.
int run_handles(const std::vector<fmg_eig_handle*>& hs,
                const std::vector<std::vector<int>>& out_index, double* lambdas,
                double* const* u_hosts, const size_t* u_lens, fmg_eig_stats* stats,
                int32_t* statuses) {
  for (size_t g = 0; g < hs.size(); ++g) {
    fmg_eig_handle* h = hs[g];
    for (int b = 0; b < h->nb; ++b) {
      const int i = out_index[g][b];
      if (u_hosts && u_hosts[i]) {
        if (!u_lens || u_lens[i] != h->L(h->probs[b].levels).g.interior()) return FMG_EINVAL;
      }
    }
  }
  // A pinned (or registered) host buffer receives the interior of u straight from the padded
  // finest level by one strided copy-engine transfer (no staging copy); pageable buffers are
  // staged in h->uout and copied.
  std::vector<std::vector<char>> pinned(hs.size());
  for (size_t g = 0; g < hs.size(); ++g) {
    fmg_eig_handle* h = hs[g];
    pinned[g].assign(h->nb, 0);
    for (int b = 0; u_hosts && b < h->nb; ++b) {
      const int i = out_index[g][b];
      cudaPointerAttributes attr;
      if (u_hosts[i] && cudaPointerGetAttributes(&attr, u_hosts[i]) == cudaSuccess &&
          attr.type == cudaMemoryTypeHost && attr.devicePointer)
        pinned[g][b] = 1;
      cudaGetLastError();
    }
  }
  for (size_t g = 0; g < hs.size(); ++g) {
    fmg_eig_handle* h = hs[g];
    cudaStream_t s = h->stream;
    CK(cudaEventRecord(h->ev0, s));
    CK(upload_params(h, s));
    CK(cudaGraphLaunch(h->exec, s));
    CK(cudaEventRecord(h->ev1, s));
    if (u_hosts) {
      bool staged = false;
      for (int b = 0; b < h->nb; ++b) {
        if (!u_hosts[out_index[g][b]]) continue;
        if (pinned[g][b]) {
          Level v = view(h->L(h->probs[b].levels), b, 1);
          CK(copy_interior_to_host(v.g, v.u, u_hosts[out_index[g][b]], s));
        } else {
          staged = true;
        }
      }
      if (staged) enqueue_outputs(h, s);
    }
    if (stats) enqueue_checks(h, s);
    h->activate(1);
  }
  int rc = FMG_OK;
  for (size_t g = 0; g < hs.size(); ++g) {
    fmg_eig_handle* h = hs[g];
    cudaStream_t s = h->stream;
    const int nb = h->nb, L = h->levels();
    std::vector<double> lam(nb), lv((size_t)L * nb), sc(3 * (size_t)nb);
    std::vector<int> st((size_t)L * nb), it((size_t)L * nb), wf(nb);
    CK(cudaMemcpyAsync(lam.data(), h->lam, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(st.data(), h->status, sizeof(int) * L * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(wf.data(), h->wait_fail, sizeof(int) * nb, cudaMemcpyDeviceToHost, s));
    if (stats) {
      CK(cudaMemcpyAsync(lv.data(), h->lam_levels, sizeof(double) * L * nb,
                         cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(it.data(), h->iters, sizeof(int) * L * nb, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(sc.data(), h->scal, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, s));
    }
    for (int b = 0; u_hosts && b < nb; ++b) {
      const int i = out_index[g][b];
      if (u_hosts[i] && !pinned[g][b])
        CK(cudaMemcpyAsync(u_hosts[i], h->uout + h->uoff[b], sizeof(double) * u_lens[i],
                           cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    for (int b = 0; b < nb; ++b) {
      const int i = out_index[g][b];
      const int lb = h->probs[b].levels;
      const int code = instance_code(st.data(), wf.data(), nb, b, lb);
      if (code == FMG_ETIMEOUT || (code == FMG_ENOCONV && rc == FMG_OK)) rc = code;
      lambdas[i] = lam[b];
      if (statuses) statuses[i] = code;
      if (stats) {
        fmg_eig_stats& o = stats[i];
        memset(&o, 0, sizeof(o));
        o.lambda = lam[b];
        o.solve_ms = ms;
        o.levels = lb;
        o.status = code;
        for (int k = 1; k <= lb; ++k) {
          o.lambda_levels[k - 1] = lv[(size_t)(k - 1) * nb + b];
          o.scf_iters[k - 1] = it[(size_t)(k - 1) * nb + b];
        }
        // b(u,u) - 1 and lambda - a(u,u) - (Wu,u) - zeta int u^4 on the finest level
        o.norm_defect = sc[nb + b] - 1.0;
        o.identity_defect = lam[b] - (sc[b] + h->probs[b].zeta * sc[2 * nb + b]);
      }
    }
  }
  return rc;
}

}  // namespace fmg

extern "C" {

const char* fmg_eig_strerror(int code) {
  switch (code) {
    case FMG_OK: return "ok";
    case FMG_EINVAL: return "invalid argument";
    case FMG_ENOMEM: return "out of device memory";
    case FMG_ENOCONV: return "nonlinear solve hit its iteration cap";
    case FMG_ECUDA: return "CUDA runtime error";
    case FMG_ETIMEOUT: return "bounded device wait gave up";
    case FMG_ENOTSUP: return "option combination not supported";
    default: return "unknown error";
  }
}

int fmg_eig_create(const fmg_eig_problem* prob, fmg_eig_handle** out) {
  if (!prob) {
    if (out) *out = nullptr;
    return FMG_EINVAL;
  }
  return create_handle(prob, 1, CreateOptions{}, out);
}

int fmg_eig_batch_create(const fmg_eig_problem* probs, int32_t count, fmg_eig_handle** out) {
  return create_handle(probs, count, CreateOptions{}, out);
}

int32_t fmg_eig_batch_count(const fmg_eig_handle* h) { return h ? h->nb : 0; }

int fmg_eig_level_tile(const fmg_eig_handle* h, int32_t level, int32_t* bx, int32_t* by) {
  if (!level_ok(h, level) || !bx || !by) return FMG_EINVAL;
  *bx = h->lv[level - 1].g.bx;
  *by = h->lv[level - 1].g.by;
  return FMG_OK;
}

size_t fmg_eig_level_size(const fmg_eig_handle* h, int32_t level) {
  if (!level_ok(h, level)) return 0;
  return h->lv[level - 1].g.interior();
}

void fmg_eig_destroy(fmg_eig_handle* h) { delete h; }

int fmg_eig_set_params(fmg_eig_handle* h, const fmg_eig_problem* prob) {
  if (!h || !prob || h->nb != 1) return FMG_EINVAL;
  const int v = validate(prob);
  if (v != FMG_OK) return v;
  const fmg_eig_problem& a = h->prob;
  if (prob->levels != a.levels || shared_key(*prob) != shared_key(a)) return FMG_EINVAL;
  // the pinned staging copy is read by the next solve's upload, in stream order
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return FMG_ECUDA;
  h->prob.w_const = prob->w_const;
  for (int d = 0; d < 3; ++d) h->prob.w_quad[d] = prob->w_quad[d];
  h->prob.zeta = prob->zeta;
  h->prob.omega = prob->omega;
  h->probs[0] = h->prob;
  fill_params(h);
  if (upload_params(h, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return FMG_ECUDA;
  enqueue_setup(h, h->stream);  // keep the component entry points' operators current
  h->activate(1);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return FMG_ECUDA;
  return FMG_OK;
}

int fmg_eig_kernel_count(const fmg_eig_handle* h) { return h ? h->kernel_nodes : 0; }

int fmg_eig_inject_alloc_failure(int64_t after) {
  g_alloc_fail_after.store(after < 0 ? -1 : (long long)after);
  return FMG_OK;
}

int fmg_eig_profile(fmg_eig_handle* h, double* ms, int32_t count) {
  if (!h || !ms || count < 1) return FMG_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return FMG_ECUDA;
  const int n = count < kProfCount ? count : kProfCount;
  for (int i = 0; i < n; ++i) {
    float t = 0.f;
    ms[i] = cudaEventElapsedTime(&t, h->prof[i][0], h->prof[i][1]) == cudaSuccess ? t : -1.0;
  }
  cudaGetLastError();
  return n;
}

int fmg_eig_solve_dev(fmg_eig_handle* h, double* lambda_dev, double* u_dev, size_t u_len,
                      void* stream) {
  if (!h || !lambda_dev || h->nb != 1) return FMG_EINVAL;
  const Level& fine = h->L(h->levels());
  if (u_dev && u_len != fine.g.interior()) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  CK(upload_params(h, s));
  CK(cudaGraphLaunch(h->exec, s));
  CK(cudaMemcpyAsync(lambda_dev, h->lam, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (u_dev) unpack_interior(fine.g, fine.u, u_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_solve(fmg_eig_handle* h, double* lambda, double* u_host, size_t u_len,
                  fmg_eig_stats* stats) {
  if (!h || !lambda || h->nb != 1) return FMG_EINVAL;
  double* const uh[1] = {u_host};
  const size_t ul[1] = {u_len};
  std::vector<fmg_eig_handle*> hs{h};
  std::vector<std::vector<int>> idx{{0}};
  return run_handles(hs, idx, lambda, u_host ? uh : nullptr, ul, stats, nullptr);
}

int fmg_eig_batch_solve(fmg_eig_handle* h, double* lambdas, double* const* u_hosts,
                        const size_t* u_lens, fmg_eig_stats* stats, int32_t* statuses) {
  if (!h || !lambdas) return FMG_EINVAL;
  std::vector<fmg_eig_handle*> hs{h};
  std::vector<std::vector<int>> idx{h->order};
  return run_handles(hs, idx, lambdas, u_hosts, u_lens, stats, statuses);
}

int fmg_eig_batch_solve_dev(fmg_eig_handle* h, double* lambdas_dev, void* stream) {
  if (!h || !lambdas_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  CK(upload_params(h, s));
  CK(cudaGraphLaunch(h->exec, s));
  gather_by_index(h->lam, h->inv_order, lambdas_dev, h->nb, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_solve_batch(const fmg_eig_problem* probs, int32_t count, double* lambdas,
                        double* const* u_hosts, const size_t* u_lens, fmg_eig_stats* stats,
                        int32_t* statuses) {
  if (!probs || count < 1 || !lambdas) return FMG_EINVAL;
  for (int i = 0; i < count; ++i) {
    const int v = validate(&probs[i]);
    if (v != FMG_OK) return v;
  }
  // group by the shared fields, keeping the callers' order inside each group
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < count; ++i) {
    bool placed = false;
    for (auto& g : groups)
      if (shared_key(probs[g[0]]) == shared_key(probs[i])) {
        g.push_back(i);
        placed = true;
        break;
      }
    if (!placed) groups.push_back({i});
  }
  std::vector<fmg_eig_handle*> hs;
  std::vector<std::vector<int>> idx;
  int rc = FMG_OK;
  for (auto& g : groups) {
    std::vector<fmg_eig_problem> ps;
    for (int i : g) ps.push_back(probs[i]);
    fmg_eig_handle* h = nullptr;
    rc = create_handle(ps.data(), (int)ps.size(), CreateOptions{}, &h);
    if (rc != FMG_OK) break;
    hs.push_back(h);
    std::vector<int> map(h->nb);
    for (int b = 0; b < h->nb; ++b) map[b] = g[h->order[b]];
    idx.push_back(map);
  }
  if (rc == FMG_OK) rc = run_handles(hs, idx, lambdas, u_hosts, u_lens, stats, statuses);
  for (fmg_eig_handle* h : hs) delete h;
  return rc;
}

// ---- component entry points (instance 0 of the handle) ------------------------------------
int fmg_eig_apply_operator(fmg_eig_handle* h, int32_t level, const double* x_dev,
                           double* y_dev, void* stream) {
  if (!level_ok(h, level) || !x_dev || !y_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  pack_interior(l.g, x_dev, l.r, s);
  lv_apply(l, l.r, l.y, s);
  unpack_interior(l.g, l.y, y_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_apply_mass(fmg_eig_handle* h, int32_t level, const double* x_dev, double* y_dev,
                       void* stream) {
  if (!level_ok(h, level) || !x_dev || !y_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  pack_interior(l.g, x_dev, l.r, s);
  lv_mass(l, l.r, l.y, s);
  unpack_interior(l.g, l.y, y_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_jacobi(fmg_eig_handle* h, int32_t level, const double* f_dev,
                   const double* x_in_dev, double* x_out_dev, void* stream) {
  if (!level_ok(h, level) || !f_dev || !x_in_dev || !x_out_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  pack_interior(l.g, f_dev, l.f, s);
  pack_interior(l.g, x_in_dev, l.r, s);
  lv_jacobi(l, l.f, l.r, l.y, false, s);
  unpack_interior(l.g, l.y, x_out_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_residual_restrict(fmg_eig_handle* h, int32_t level, const double* f_dev,
                              const double* x_dev, double* rc_dev, void* stream) {
  if (!level_ok(h, level) || level < 2 || !f_dev || !x_dev || !rc_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  Level& lc = h->L(level - 1);
  pack_interior(l.g, f_dev, l.f, s);
  pack_interior(l.g, x_dev, l.z, s);
  lv_residual(l, l.f, l.z, l.r, s);
  lv_restrict(l, lc, l.r, lc.y, s);
  unpack_interior(lc.g, lc.y, rc_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_prolong_add(fmg_eig_handle* h, int32_t level, const double* ec_dev, double* x_dev,
                        void* stream) {
  if (!level_ok(h, level) || level < 2 || !ec_dev || !x_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  Level& lc = h->L(level - 1);
  pack_interior(lc.g, ec_dev, lc.y, s);
  pack_interior(l.g, x_dev, l.y, s);
  lv_prolong(l, lc, lc.y, l.y, true, nullptr, nullptr, 0, s);
  unpack_interior(l.g, l.y, x_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_nonlinear_load(fmg_eig_handle* h, int32_t level, const double* u_dev,
                           double* n_dev, void* stream) {
  if (!level_ok(h, level) || !u_dev || !n_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  pack_interior(l.g, u_dev, l.r, s);
  lv_nload(l, l.r, l.y, s);
  unpack_interior(l.g, l.y, n_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_aux_rhs(fmg_eig_handle* h, int32_t level, double lambda, const double* u_dev,
                    double* f_dev, void* stream) {
  if (!level_ok(h, level) || !u_dev || !f_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  CK(cudaStreamSynchronize(s));
  double* lam_tmp = h->scal + 3 * (size_t)h->nb;
  CK(cudaMemcpy(lam_tmp, &lambda, sizeof(double), cudaMemcpyHostToDevice));
  pack_interior(l.g, u_dev, l.r, s);
  lv_rhs(l, lam_tmp, h->dparams, l.r, l.y, s);
  if (h->literal()) lv_sub_wmass(l, l.r, l.y, s);
  unpack_interior(l.g, l.y, f_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_multigrid(fmg_eig_handle* h, int32_t level, const double* f_dev, double* x_dev,
                      void* stream) {
  if (!level_ok(h, level) || !f_dev || !x_dev) return FMG_EINVAL;
  cudaStream_t s = pick(h, stream);
  h->activate(1);
  Level& l = h->L(level);
  pack_interior(l.g, f_dev, l.f, s);
  pack_interior(l.g, x_dev, l.x, s);
  enqueue_multigrid(h, level, s, false);
  unpack_interior(l.g, l.x, x_dev, s);
  CK(cudaGetLastError());
  return FMG_OK;
}

int fmg_eig_correction(fmg_eig_handle* h, int32_t level, double lambda_in,
                       const double* u_in_dev, double* lambda_out, double* u_out_dev,
                       double* u_tilde_dev, int32_t* iters) {
  if (!level_ok(h, level) || level < 2 || !u_in_dev || !lambda_out || !u_out_dev)
    return FMG_EINVAL;
  cudaStream_t s = h->stream;
  h->activate(1);
  Level& l = h->L(level);
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(h->lam, &lambda_in, sizeof(double), cudaMemcpyHostToDevice));
  pack_interior(l.g, u_in_dev, l.u, s);
  enqueue_correction(h, level, s);
  unpack_interior(l.g, l.u, u_out_dev, s);
  if (u_tilde_dev) unpack_interior(l.g, l.x, u_tilde_dev, s);
  int st = 0, it = 0;
  const size_t row = (size_t)(level - 1) * h->nb;
  CK(cudaMemcpyAsync(lambda_out, h->lam, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, h->status + row, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&it, h->iters + row, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  return st == 0 ? FMG_OK : FMG_ENOCONV;
}

int fmg_eig_augmented_system(fmg_eig_handle* h, int32_t level, const double* u_tilde_dev,
                             const double* c_host, int32_t n, double* K_host, double* M_host,
                             double* G_host) {
  if (!level_ok(h, level) || level < 2 || !u_tilde_dev || !c_host || !K_host || !M_host ||
      !G_host || n != h->nh + 1)
    return FMG_EINVAL;
  cudaStream_t s = h->stream;
  h->activate(1);
  Level& l = h->L(level);
  const size_t nn = (size_t)n * n;
  double* kd = h->kscratch;
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(kd + 3 * nn, c_host, n * sizeof(double), cudaMemcpyHostToDevice));
  pack_interior(l.g, u_tilde_dev, l.x, s);
  enqueue_augment(h, level, l.x, s);
  DenseProblem d = dense_augmented(h);
  d.c_init = kd + 3 * nn;
  d.K_out = kd;
  d.M_out = kd + nn;
  d.G_out = kd + 2 * nn;
  d.iters_out = h->iters;
  d.status_out = h->status;
  dense_scf(d, 1, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(K_host, kd, nn * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(M_host, kd + nn, nn * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(G_host, kd + 2 * nn, nn * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return FMG_OK;
}

int fmg_eig_coarse_solve(fmg_eig_handle* h, double* lambda_out, double* u_dev, int32_t* iters) {
  if (!h || !lambda_out || !u_dev) return FMG_EINVAL;
  cudaStream_t s = h->stream;
  h->activate(1);
  enqueue_coarse(h, s);
  unpack_interior(h->L(1).g, h->L(1).u, u_dev, s);
  int st = 0, it = 0;
  CK(cudaMemcpyAsync(lambda_out, h->lam, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&it, h->iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  return st == 0 ? FMG_OK : FMG_ENOCONV;
}

}  // extern "C"
