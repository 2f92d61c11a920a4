// Engine internals shared by the C ABI (fmg_api.cu) and the request server (serve.cu): the
// level hierarchy of a handle, the handle itself, and the calls that build and run it.
//
// A handle holds a batch of nb instances (nb = 1 for fmg_eig_create) sorted by level count,
// largest first.  Level k's arrays hold the cnt[k] instances that have a level k back to
// back, so on the FMG stage of level k the active instances are 0 .. cnt[k] - 1 of every
// array and each step of the stage is one launch over all of them (Grid::nb).
#pragma once

#include <algorithm>
#include <functional>
#include <new>
#include <vector>

#include "fmg_internal.h"

namespace fmg {

struct Level {
  Grid g;
  int cap = 0;  // instances allocated (cnt[k])
  Coef2D c{};   // operator of the auxiliary problem (A + W, or A in the paper-literal form)
  Coef3D c3{};
  Coef2D cw{};  // A + W (the same arrays as c unless the form is paper-literal)
  Coef3D cw3{};
  double *x = nullptr, *xt = nullptr, *f = nullptr, *r = nullptr, *u = nullptr,
         *y = nullptr, *z = nullptr;
  Density2D b{};          // density stencil of u~ (augmented pass), 2D
  Density3D b3{};         // same, 3D
  // mixed precision: FP32 coefficient tables and single-precision V-cycle vectors
  CoefT ct{};
  float *x32 = nullptr, *xt32 = nullptr, *f32 = nullptr, *r32 = nullptr;
  // mixed precision: double-float split (hi + lo) of the vector the nonlinear kernels read
  float *uhi = nullptr, *ulo = nullptr;
  // mixed precision, large 2D levels: tensor maps of the two x buffers (tile + halo box) and
  // of f32 (tile box) for the TMA-fed sweeps; tm_base[q] is the buffer tm_x[q] describes
  bool tma = false;
  const float* tm_base[2] = {};
  TMAMap tm_x[2]{}, tm_f{};
  double* pw = nullptr;   // (x / r)^m table for the 2D T3 sums (levels >= 2)
  double* t3map = nullptr;  // class sums -> T3 map of this level (levels >= 2)
};

// The same level restricted to instances first .. first + count - 1.
Level view(const Level& l, int first, int count);

enum ProfId { kProfJacobi, kProfResidual, kProfRestrict, kProfProlong, kProfRhs,
              kProfMoments, kProfDense, kProfVcycle, kProfT3, kProfCoef, kProfCount };

// How a handle is built.  The C ABI handles record the whole solve as one CUDA graph and
// keep operators for the component entry points; the server's cohorts launch directly (with
// an event after every FMG stage), allocate stream-ordered from the device's memory pool (so
// releasing a finished cohort does not wait for the others) and only reuse tuned tiles.
struct CreateOptions {
  bool graph = true;            // capture the solve as a CUDA graph
  bool component_setup = true;  // operators ready for the component entry points
  bool async_alloc = false;     // cudaMallocAsync / cudaFreeAsync on the handle's stream
  int tune = 2;                 // 0: default tiles, 1: tuned tiles from the cache only, 2: tune
  // When set (nb pinned doubles owned by the caller): after the coarse solve and after each
  // finer FMG stage, the solve copies the eigenvalues of the instances that finish there to
  // stage_lam[first..] and records one of the handle's stage events (inside the graph too).
  double* stage_lam = nullptr;
};

// Test hook behind fmg_eig_inject_alloc_failure: true when the device allocation about to
// be made is the one chosen to fail (each call counts one allocation).
bool injected_alloc_failure();

}  // namespace fmg

struct fmg_eig_handle {
  fmg_eig_problem prob{};  // settings shared by the batch; levels = the largest instance's
  int nb = 1;              // instances
  std::vector<fmg_eig_problem> probs;  // per instance, sorted by level count (descending)
  std::vector<int> order;              // order[b]: caller's index of sorted instance b
  std::vector<int> cnt;                // cnt[k], k = 1..levels (+ cnt[levels + 1] = 0)
  std::vector<size_t> uoff;            // offset of sorted instance b's output in uout
  fmg::CreateOptions opt;
  int dev = 0;
  cudaStream_t stream = nullptr;
  // Independent branches of a solve run on side streams, forked from and joined back to the
  // solve's stream with events (inside a capture they become parallel graph branches): the
  // two side chains of the augmented pass (side 0, 1) and the operator setup of levels >= 2
  // (side 2, joined at the stage that first needs the level).
  cudaStream_t side[3] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {}, ev_level[FMG_MAX_LEVELS + 1] = {};
  bool level_pending[FMG_MAX_LEVELS + 1] = {};  // enqueue-time: setup of level k not joined yet
  std::vector<fmg::Level> lv;  // lv[0] = level 1
  std::vector<void*> allocs;
  size_t bytes = 0;  // device bytes allocated
  bool dry = false;  // count the bytes of every allocation without allocating
  int nh = 0, ntri = 0, nvert = 3, maxadj = 6;
  double tri_vol = 0.0;
  // per-instance arrays (sorted order): L1, M1, L1inv nh*nh; c, cstart nh + 1; scalars 1
  // L1 = A + W on level 1 (the small nonlinear solves), L1A the operator whose inverse is the
  // coarsest V-cycle solve (the same array unless the form is paper-literal)
  double *L1 = nullptr, *L1A = nullptr, *M1 = nullptr, *L1inv = nullptr;
  int *tri = nullptr, *adj = nullptr;
  int npat = 0;  // gather lists of the dense G(c) assembly (DenseProblem)
  int *gent = nullptr, *gstart = nullptr, *gidx = nullptr;
  double *lam = nullptr, *c = nullptr, *cstart = nullptr, *auu = nullptr, *buu = nullptr,
         *partials = nullptr, *partials2 = nullptr, *t3 = nullptr, *t3_partials = nullptr, *gAd = nullptr,
         *gMd = nullptr, *t1d = nullptr, *B1d = nullptr, *t0 = nullptr,
         *lam_levels = nullptr, *scal = nullptr, *kscratch = nullptr, *uout = nullptr;
  double* cg = nullptr;  // conjugate gradient smoother: r.r (2 slots) and p.L p per instance
  int *iters = nullptr, *status = nullptr;  // [level][instance]
  int* wait_fail = nullptr;  // [instance]: 1 when a bounded device wait gave up in the solve
  int* inv_order = nullptr;                 // sorted index of the caller's instance i
  // device copy read by the kernels (nparams), and its pinned host staging uploaded at every
  // solve; the paper-literal form keeps nb more entries with the form set to W_LEFT, from
  // which the A + W coefficients are built (dparams_full)
  int nparams = 1;
  fmg::PotentialParams* dparams = nullptr;
  fmg::PotentialParams* dparams_full = nullptr;
  fmg::PotentialParams* hparams = nullptr;
  bool literal() const { return prob.operator_form == FMG_PAPER_LITERAL; }
  bool mixed() const { return prob.precision != FMG_FP64; }
  bool bf16() const { return prob.precision == FMG_MIXED_BF16; }
  // profiling: event pairs around the first finest-level launch of each profiled step
  cudaEvent_t prof[fmg::kProfCount][2] = {};
  bool prof_armed[fmg::kProfCount] = {};
  int kernel_nodes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // stage marks (CreateOptions::stage_lam): event and sorted instance range per mark
  struct StageMark {
    cudaEvent_t ev;
    int first, count;
  };
  std::vector<StageMark> marks;
  size_t dense_smem = 0;

  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    const size_t nbytes = std::max<size_t>(count, 1) * sizeof(T);
    if (dry) {
      bytes += (nbytes + 511) / 512 * 512;
      return nullptr;
    }
    if (fmg::injected_alloc_failure()) throw std::bad_alloc();
    const cudaError_t e = opt.async_alloc ? cudaMallocAsync(&p, nbytes, stream)
                                          : cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    allocs.push_back(p);
    bytes += nbytes;
    cudaMemsetAsync(p, 0, nbytes, stream);
    return static_cast<T*>(p);
  }
  ~fmg_eig_handle();
  fmg::Level& L(int k) { return lv[k - 1]; }
  int levels() const { return prob.levels; }
  // every level launches over `count` instances (the active prefix of the stage)
  void activate(int count) {
    for (fmg::Level& l : lv) l.g.nb = std::min(count, l.cap);
  }
};

namespace fmg {

int validate(const fmg_eig_problem* p);
bool same_shared_settings(const fmg_eig_problem& a, const fmg_eig_problem& b);
int create_handle(const fmg_eig_problem* probs, int count, const CreateOptions& opt,
                  fmg_eig_handle** out);
// Device bytes create_handle will allocate for these instances (an upper bound).
size_t estimate_bytes(const fmg_eig_problem* probs, int count);
// The whole of Algorithm 3.2 for every instance, in stream order on s.  after_stage, when
// given, is called once the work of the coarse solve (k = 1) and of each finer FMG stage k
// is enqueued, with the sorted instances [first, first + count) whose last level is k.
using StageHook = std::function<void(int k, int first, int count)>;
void enqueue_fmg(fmg_eig_handle* h, cudaStream_t s, const StageHook* after_stage = nullptr);
// host staging of the per-instance parameters from h->probs (before an upload)
void fill_params(fmg_eig_handle* h);
// upload the host staging of the parameters (every solve starts with it)
cudaError_t upload_params(fmg_eig_handle* h, cudaStream_t s);
// every instance's u from its finest level into h->uout (interior layout)
void enqueue_outputs(fmg_eig_handle* h, cudaStream_t s);
// FMG_OK, FMG_ENOCONV or FMG_ETIMEOUT for sorted instance b with lb levels, from the copied
// statuses st[level][instance] (nb per level) and wait words of a solve
int instance_code(const int* st, const int* wait_fail, int nb, int b, int lb);

}  // namespace fmg
