// Internal declarations shared by the CUDA translation units of libfmg_eig.
//
// Device layout of a level vector (2D): the (n+1) x (n+1) grid of ALL nodes, boundary
// included, row-major with x fastest and a row pitch of `pitch` elements (a multiple of 32).
// Boundary entries and the pitch padding are zero and are never written, so stencils need no
// boundary branches.  3D adds planes of (n+1) rows each.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fmg_eig.h"

namespace fmg {

// Batched launches: every per-level array holds its instances back to back, instance b's
// vector starting at element b * stride; every launcher runs instances 0 .. nb - 1 of the
// arrays it is given, and per-instance scalars (lambda, parameters, dots) are indexed by b.
struct Grid {
  int dim = 2;
  int n = 0;          // cells per side
  int pitch = 0;      // elements per row
  int rows = 0;       // rows per plane (n + 1)
  size_t stride = 0;  // elements per vector of one instance
  double h = 0;
  int nb = 1;         // instances of a launch
  int bx = 32, by = 8;  // thread-block shape of the stencil kernels on this level
  bool walk_all = false;  // FP64 cubic-load kernels as walks whatever the launch size
  size_t interior() const {
    size_t m = (size_t)(n - 1);
    return dim == 2 ? m * m : m * m * m;
  }
};

// A vector split into double-float halves (hi + lo, FP32 each) for the nonlinear kernels of
// the mixed-precision modes, which compute in double-float arithmetic on the FP32 pipes.
// up to two vectors restricted by one launch
struct RestrictVecs {
  const double* rf[2];
  double* rc[2];
};

struct SplitVec {
  const float* hi;
  const float* lo;
};

// Stencil coefficients of L = A + W on one 2D level (see grid2d.cu for the closed forms).
struct Coef2D {
  double* cC;    // diagonal
  double* cE;    // coupling (i,j)-(i+1,j)
  double* cN;    // coupling (i,j)-(i,j+1)
  double* cNE;   // coupling (i,j)-(i+1,j+1)
  double* dinv;  // omega / cC
  double* tab;   // 8 * (n + 1) separable parts of the coefficients (setup scratch)
};

// Problem parameters that may change between solves of one handle.  They live in device
// memory (uploaded at the start of every solve), so kernels take a device pointer to them.
struct PotentialParams {
  double w0, wx, wy, wz;
  double zeta;
  double omega;
  int operator_form;
  int pad;
};

// ---- 2D level kernels (grid2d.cu) -------------------------------------------------------
void coef2d_setup(const Grid& g, const PotentialParams* p_dev, const Coef2D& c, cudaStream_t s);
void apply2d(const Grid& g, const Coef2D& c, const double* x, double* y, cudaStream_t s);
void mass2d(const Grid& g, const double* x, double* y, cudaStream_t s);
// the same from the double-float split of x (mixed-precision modes)
void mass2d_df(const Grid& g, SplitVec x, double* y, cudaStream_t s);
// f -= W u, W u = (A + W) u - A u from the coefficient sets cw (A + W) and ca (A)
void sub_wmass2d(const Grid& g, const Coef2D& cw, const Coef2D& ca, const double* u, double* f,
                 cudaStream_t s);
void jacobi2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* xo,
              bool x_is_zero, cudaStream_t s);
void residual2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* r,
                cudaStream_t s);
// Chebyshev step: d = (first ? 0 : alpha d) + beta D^{-1} (f - L x), xo = x + d (x = 0 when
// x_zero); needs the coefficients built with omega = 1 (dinv = 1/D)
void cheb2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* d,
            double* xo, double alpha, double beta, bool first, bool x_zero, cudaStream_t s);
// rc = P^T rf; with rf2 given, also rc2 = P^T rf2 in the same launch
void restrict2d(const Grid& fine, const Grid& coarse, const double* rf, double* rc,
                cudaStream_t s, const double* rf2 = nullptr, double* rc2 = nullptr);
// xf = (add ? xf : 0) + P ec (+ scale[b * scale_stride] * extra for instance b when extra is
// given)
void prolong2d(const Grid& fine, const Grid& coarse, const double* ec, double* xf, bool add,
               const double* extra, const double* scale, int scale_stride, cudaStream_t s);
void nload2d(const Grid& g, const double* u, double* out, cudaStream_t s);
// f = lam[b] * M u - p[b].zeta * N(u) for instance b
void rhs2d(const Grid& g, const double* lam, const PotentialParams* p_dev, const double* u,
           double* f, cudaStream_t s);
// the same right-hand side evaluated in FP32 (mixed-precision iteration), stored in FP64
void rhs2d_f32(const Grid& g, const double* lam, const PotentialParams* p_dev, const double* u,
               double* f, cudaStream_t s);
// the same right-hand side in double-float arithmetic from the split u (mixed-precision modes)
void rhs2d_df(const Grid& g, const double* lam, const PotentialParams* p_dev, SplitVec u,
              double* f, cudaStream_t s);
// Dense level-1 matrices L_1 and M_1 (n1-1)^2 square, row-major, interior numbering (one
// pair per instance, back to back).
void dense_level1_2d(const Grid& g, const Coef2D& c, double* L, double* M, cudaStream_t s);
// sin-product start vector for the level-1 nonlinear solve (instance b at c + b * cstride)
void start_vector(const Grid& g, double* c, int cstride, cudaStream_t s);

// ---- 3D level kernels (grid3d.cu) -------------------------------------------------------
// Couplings of L on the Kuhn mesh: a[0] diagonal, a[1 + d] the coupling of p with p + d for
// d = X, Y, Z, XY, XZ, YZ, XYZ (the coupling with p - d is a[1 + d] at p - d).
struct Coef3D {
  double* a[8];
  double* dinv;  // omega / diagonal
  double* tab;   // 15 * (n + 1) separable parts (setup scratch)
};
struct Density3D {
  double* a[8];  // same layout as Coef3D::a
};
struct Stencil15 {
  const double* a[8];
};
void coef3d_setup(const Grid& g, const PotentialParams* p_dev, const Coef3D& c, cudaStream_t s);
void apply3d(const Grid& g, const Coef3D& c, const double* x, double* y, cudaStream_t s);
void mass3d(const Grid& g, const double* x, double* y, cudaStream_t s);
void mass3d_df(const Grid& g, SplitVec x, double* y, cudaStream_t s);
void sub_wmass3d(const Grid& g, const Coef3D& cw, const Coef3D& ca, const double* u, double* f,
                 cudaStream_t s);
void jacobi3d(const Grid& g, const Coef3D& c, const double* f, const double* x, double* xo,
              bool x_is_zero, cudaStream_t s);
void residual3d(const Grid& g, const Coef3D& c, const double* f, const double* x, double* r,
                cudaStream_t s);
void cheb3d(const Grid& g, const Coef3D& c, const double* f, const double* x, double* d,
            double* xo, double alpha, double beta, bool first, bool x_zero, cudaStream_t s);
void restrict3d(const Grid& fine, const Grid& coarse, const double* rf, double* rc,
                cudaStream_t s, const double* rf2 = nullptr, double* rc2 = nullptr);
void prolong3d(const Grid& fine, const Grid& coarse, const double* ec, double* xf, bool add,
               const double* extra, const double* scale, int scale_stride, cudaStream_t s);
void nload3d(const Grid& g, const double* u, double* out, cudaStream_t s);
void rhs3d(const Grid& g, const double* lam, const PotentialParams* p_dev, const double* u,
           double* f, cudaStream_t s);
void rhs3d_f32(const Grid& g, const double* lam, const PotentialParams* p_dev, const double* u,
               double* f, cudaStream_t s);
void nload_density3d(const Grid& g, const double* u, double* nl, const Density3D& b,
                     cudaStream_t s);
// double-float versions from the split u (mixed-precision modes)
void rhs3d_df(const Grid& g, const double* lam, const PotentialParams* p_dev, SplitVec u,
              double* f, cudaStream_t s);
// (the _df versions write the density stencil as double-float splits: see put_entry)
void nload_density3d_df(const Grid& g, SplitVec u, double* nl, const Density3D& b,
                        cudaStream_t s);
void coarsen_density3d(const Grid& fine, const Grid& coarse, const Density3D& bf,
                       const Density3D& bc, cudaStream_t s, bool split = false);
void dense_level1_3d(const Grid& g, const Coef3D& c, double* L, double* M, cudaStream_t s);
void density_dense3d(const Grid& g, const Density3D& b, double* B, cudaStream_t s,
                     bool split = false);
void gather_vec3d(const Grid& g, const double* a, const double* b, const double* c, double* oa,
                  double* ob, double* oc, cudaStream_t s);
void start_vector3d(const Grid& g, double* c, int cstride, cudaStream_t s);

// ---- 3D augmented pass (augment3d.cu) -----------------------------------------------------
// T3 per coarse Kuhn tetrahedron (20 per tetrahedron, sorted triples of its 4 vertices;
// partials: t3_partials3d doubles per instance, t3: 20 per tetrahedron per instance),
// tetrahedron index 6 * (I + n1 (J + n1 L)) + s, s the axis permutation in lexicographic
// order, vertices (V, V + e_s0, V + e_s0 + e_s1, V + (1,1,1)).
size_t t3_partials3d(const Grid& fine, int n1);
// pw: the level's (x/r)^m table (t3_power_table)
void t3_moments3d(const Grid& fine, int n1, const double* u, const double* pw,
                  const double* map, double* partials, double* t3, cudaStream_t s);
void t3_map3d(int r, double* out);  // 20 * 15 * 20 doubles

// ---- Mixed precision (mixed.cu) ------------------------------------------------------------
// FP32 separable coefficient tables of one level for the single-precision V-cycle: tab =
// the level's FP64 tables (2D: 8, 3D: 15 per instance, n + 1 entries each) rounded to FP32
// and tablo their remainders (tab + tablo is their double-float split); cst = kCst floats
// per instance: the 3D constants (C, axis, face, body) at 0..3 with their remainders at
// kCstLo + 0..3, and omega at kCstOmega with its remainder at kCstOmegaLo.
struct CoefT {
  float* tab;
  float* tablo;
  float* cst;
};
// 3D single-precision sweeps: coupling = ((x part + y part) + z part) + class constant, the
// large constant (6h, -h) added last so that each coefficient is one rounding from its FP64
// value.  (Adding the constant first and three rounded table entries after it left the
// smooth-mode part of the operator off by several roundings of the constant, which showed
// as |d lambda| up to 3e-8 on strongly nonlinear 3D problems.)
constexpr int kCst = 16;
constexpr int kCstOmega = 4;
constexpr int kCstOmegaLo = 5;
constexpr int kCstLo = 8;

// hi[i] + lo[i] = u[i] to 2^-47 relative (hi: u[i]'s significand cut to 24 bits), i < n;
// n even, the arrays allocation-aligned
void split_df(const double* u, float* hi, float* lo, size_t n, cudaStream_t s);
// Storage of the single-precision V-cycle arrays (the float* below): FP32, or bfloat16 when
// `bf` is set (FMG_MIXED_BF16; arithmetic stays FP32).  Bytes per element:
size_t mixed_elem_bytes(bool bf16_storage);
// contiguous conversions over n entries (all instances of a level at once)
void add_f32(const float* e, double* x, size_t n, cudaStream_t s, bool bf = false);  // x += e
// r = f - L x with the FP64 operator of the level (2D uses c2, 3D c3), stored single
void residual_mixed(const Grid& g, const Coef2D& c2, const Coef3D& c3, const double* f,
                    const double* x, float* r, cudaStream_t s, bool bf = false);
// the split tables and constants of level g from its FP64 tables (c2.tab / c3.tab written)
void tables_f32(const Grid& g, const Coef2D& c2, const Coef3D& c3,
                const PotentialParams* pp, const CoefT& ct, cudaStream_t s);
// TMA-fed single-precision sweeps of the large levels (sweep_tma.cu).  A TMAMap holds a
// tensor map (CUtensorMap) of one level vector: columns, rows and instances, with a box of
// one tile (halo = true: the x box, 2 rows taller).
struct TMAMap {
  alignas(64) unsigned char bytes[128];
};
constexpr int kTMAMinCells2 = 512;  // 2D levels with n >= this use the TMA sweeps
constexpr int kTMAMinCells3 = 128;  // 3D levels likewise
bool tma_sweep_applies(const Grid& g);
bool encode_level_map(const Grid& g, int cap, const float* base, bool bf, bool halo,
                      TMAMap* out);
// mode 0: residual y = f - L x; 1: Jacobi y = x + omega D^-1 (f - L x); 2: Jacobi from x = 0.
// A tile wait that runs out sets wait_fail[b] = 1 for its instance b (wait_fail: g.nb ints);
// `expire` makes every tile wait give up at once (the FMG_FLAG_EXPIRE_WAITS test hook).
void sweep32_tma(const Grid& g, const CoefT& ct, const TMAMap& mx, const TMAMap& mf, float* y,
                 int mode, int* wait_fail, bool expire, cudaStream_t s, bool bf = false);
// damped Jacobi sweep / residual with coefficients rebuilt from the FP32 tables
void jacobi32(const Grid& g, const CoefT& ct, const float* f, const float* x, float* xo,
              bool zero, cudaStream_t s, bool bf = false);
void residual32(const Grid& g, const CoefT& ct, const float* f, const float* x, float* r,
                cudaStream_t s, bool bf = false);
void restrict32(const Grid& fine, const Grid& coarse, const float* rf, float* rc,
                cudaStream_t s, bool bf = false);
void prolong32_add(const Grid& fine, const Grid& coarse, const float* ec, float* xf,
                   cudaStream_t s, bool bf = false);
void coarse32(const Grid& g, const double* Linv, const float* x, float* y, cudaStream_t s,
              bool bf = false);
// The levels of a single-precision V-cycle below the TMA-fed ones (vcycle32_mid.cu), two
// kernels per level, bit-identical to the separate sweep, residual and transfer kernels:
//   down: xo = nu_pre Jacobi sweeps from x = 0 on L(g) x = f, rc = P^T (f - L xo);
//   up:   xo = nu_post Jacobi sweeps from x + P ec (xo and x distinct).
// They take 2D levels of up to kMid32MaxCells cells per side with at most 4 + 4 sweeps, and
// 3D levels of up to kMid32MaxCells3 with at most 2 + 2.
constexpr int kMid32MaxCells = 256;
constexpr int kMid32MaxCells3 = 32;  // measured: 64 no faster than the separate kernels
bool vcycle32_mid_applies(const Grid& g, int nu_pre, int nu_post);
void vcycle32_down(const Grid& g, const CoefT& ct, const Grid& gc, const float* f, float* xo,
                   float* rc, int nu_pre, cudaStream_t s, bool bf = false);
void vcycle32_up(const Grid& g, const CoefT& ct, const Grid& gc, const float* f,
                 const float* x, float* xo, const float* ec, int nu_post, cudaStream_t s,
                 bool bf = false);

// ---- Reductions (reduce.cu) -------------------------------------------------------------
// out[b] = sum_i a[b vst + i] * b[b vst + i] over n entries for instances b < nb;
// deterministic two-stage tree whose order depends on n only.  `partials` holds
// nb * kReduceBlocks doubles.
constexpr int kReduceBlocks = 1024;
void dot(const double* a, const double* b, size_t n, double* partials, double* out,
         cudaStream_t s, int nb = 1, size_t vst = 0);
// Conjugate gradient smoother steps over nb instances of `stride` elements (n = nb stride):
// x += a p, r -= a q with a = rr[b] / pq[b]; then p = r + (rr_new[b] / rr_old[b]) p
void cg_update(size_t n, size_t stride, const double* rr, const double* pq, const double* p,
               const double* q, double* x, double* r, cudaStream_t s);
void cg_direction(size_t n, size_t stride, const double* rr_new, const double* rr_old,
                  const double* r, double* p, cudaStream_t s);

// ---- Interior <-> padded packing (pack.cu) ----------------------------------------------
// (instance b: interior vector at b * g.interior(), padded one at b * g.stride)
void pack_interior(const Grid& g, const double* interior, double* padded, cudaStream_t s);
void unpack_interior(const Grid& g, const double* padded, double* interior, cudaStream_t s);
// The interior of one instance's padded vector into a pinned host buffer by one strided
// copy-engine transfer (2D: a pitched 2D copy, 3D: a pitched 3D copy), no staging buffer.
cudaError_t copy_interior_to_host(const Grid& g, const double* padded, double* host,
                                  cudaStream_t s);
// dst[i] = src[idx[i]], i < n
void gather_by_index(const double* src, const int* idx, double* dst, int n, cudaStream_t s);
// padded level-1 vectors from dense coefficient vectors c (instance b at c + b * cstride)
void scatter_level1(const Grid& g, const double* c, size_t cstride, double* padded,
                    cudaStream_t s);

// ---- Augmented-space fine pass (augment2d.cu) ---------------------------------------------
// Density stencil B(u)_pq = int u^2 phi_p phi_q of one 2D level (couplings to p, E, N, NE).
struct Density2D {
  double *C, *E, *N, *NE;
};
// nl = N(u) (int u^3 phi_p) and the density stencil of u on level g, in one pass.
void nload_density2d(const Grid& g, const double* u, double* nl, const Density2D& b,
                     cudaStream_t s);
void nload_density2d_df(const Grid& g, SplitVec u, double* nl, const Density2D& b,
                        cudaStream_t s);
// Galerkin coarsening of the density stencil: bc = P^T bf P.
// split: the entries are stored as double-float splits (mixed modes; see nload_density*_df)
void coarsen_density2d(const Grid& fine, const Grid& coarse, const Density2D& bf,
                       const Density2D& bc, cudaStream_t s, bool split = false);
// T3^T_abc = int_T u mu_a mu_b mu_c per coarse triangle (10 per triangle, a <= b <= c,
// lexicographic), from per-class monomial sums.  pw: (x/r)^m table of the level, map: the
// level's 2 x 10 x 25 map (t3_map2d), partials: t3_partials2d(fine, n1) doubles.
size_t t3_partials2d(const Grid& fine, int n1);
void t3_moments2d(const Grid& fine, int n1, const double* u, const double* pw,
                  const double* map, double* partials, double* t3, cudaStream_t s);
void t3_class_moments2d(double out[2 * 7 * 10]);
void t3_map2d(int r, double out[2 * 10 * 25]);
void t3_power_table(int r, double* out);  // 4 * (r + 1) doubles
// dense level-1 data for the augmented solve: gA, gM, t1 (nh) and B1 (nh x nh) from padded
// level-1 vectors and the level-1 density stencil (per instance, back to back)
void gather_level1_2d(const Grid& g1, const double* gA_pad, const double* gM_pad,
                      const double* t1_pad, const Density2D& b1, double* gA, double* gM,
                      double* t1, double* B1, cudaStream_t s, bool split = false);

// ---- Dense small solves (dense.cu) -------------------------------------------------------
// A batch of problems shares the geometry (tri, adj) and keeps the per-instance arrays
// back to back: L1, M1, B1 nh*nh; gA, gM, t1 nh; t3 ntri*nt3; c_init, c_out nh + 1;
// auu, buu, t0, lam_out, iters_out, status_out and params one each.
struct DenseProblem {
  int nh;              // coarse unknowns (interior nodes of level 1)
  int aug;             // 1: basis (phi^H, u~), n = nh + 1; 0: basis phi^H, n = nh
  int ntri;            // coarse simplices
  int nvert;           // vertices per simplex (3 in 2D, 4 in 3D)
  int nt3;             // entries of T3 per simplex (10 in 2D, 20 in 3D)
  const int* tri;      // ntri * nvert coarse interior indices, -1 on the boundary
  const int* adj;      // nh * maxadj codes (simplex << 3 | local vertex), -1 terminated
  int maxadj;
  // Gather lists of the coarse block of G(c) (optional; nullptr: walk the adjacency): the
  // npat structurally nonzero entries gent[q] = a nh + b, and for each the simplex-local
  // indices gidx[gstart[q] .. gstart[q + 1]) = t (nvert + 1)^2 + la (nvert + 1) + lb of the
  // simplices t around a (adjacency order, then vertex order) with vertex lb = b.
  int npat;
  const int* gent;
  const int* gstart;
  const int* gidx;
  double tri_vol;      // |T|
  double quart_off;    // |T| 2 d! / (d + 4)!, d = nvert - 1 (int_T w^2 mu_a mu_b / h_2)
  const double* L1;    // nh*nh, operator of level 1
  const double* M1;    // nh*nh, mass of level 1
  // augmented problem only:
  const double* gA;    // nh: P^T..P^T L u~
  const double* gM;    // nh: P^T..P^T M u~
  const double* t1;    // nh: int u~^3 phi^H_a
  const double* B1;    // nh*nh: int u~^2 phi^H_a phi^H_b
  const double* t3;    // ntri * nt3: int_T u~ mu_a mu_b mu_c (sorted triples)
  const double* auu;   // u~^T L u~
  const double* buu;   // u~^T M u~
  const double* t0;    // int u~^4
  const PotentialParams* params;  // device; zeta read from here
  double tol;
  int max_iter;
  const double* c_init;  // nullptr: augmented start e_u / sqrt(buu); level-1: caller fills
  double* c_out;         // n
  double* lam_out;       // 1
  int* iters_out;        // 1
  int* status_out;       // 1 (0 converged, 1 cap hit)
  // optional (a single problem only): assemble K0, M, G(c_init) into these n x n outputs
  double* K_out;
  double* M_out;
  double* G_out;
};
constexpr size_t kDenseSmemLimit = 200 * 1024;  // dynamic shared memory of the dense solve
size_t dense_smem_bytes(int n, int ntri, int nvert, int aug);
cudaError_t dense_prepare(size_t max_smem);  // opt in to large dynamic shared memory
void dense_scf(const DenseProblem& p, int nb, cudaStream_t s);  // one CTA per problem
// Linv = L^{-1} for SPD n x n matrices (LDL^T), one CTA per instance.
void dense_spd_inverse(const double* L, double* Linv, int n, int nb, cudaStream_t s);
// y(padded level 1) = Linv * x(padded level 1) on the interior nodes (2D or 3D)
void coarse_matvec(const Grid& g, const double* Linv, const double* x, double* y,
                   cudaStream_t s);

// ---- the small levels of a 2D V-cycle in one kernel (vcycle_small.cu) ---------------------
constexpr int kSmallMaxLevels = 6;    // entry level and the levels below it
constexpr int kSmallMaxCells = 32;    // cells per side of the entry level
constexpr size_t kSmallSmemLimit = 96 * 1024;
struct SmallLevel2D {
  int n, pitch;
  size_t stride;
  Coef2D c;  // the V-cycle's operator on this level
};
struct SmallVcycle {
  int levels;  // the entry level; levels 1 .. levels take part
  int nu_pre, nu_post, x_zero;
  SmallLevel2D lv[kSmallMaxLevels];  // level j at index j - 1
  const double* Linv;                // level-1 inverse, nh x nh per instance
  const double* f;                   // the entry level's right-hand side (batched arrays)
  double* x;                         // the entry level's iterate, read unless x_zero
};
size_t vcycle_small_smem(const SmallVcycle& v);
// One V-cycle from the entry level for instances 0 .. nb - 1; an error (before launching)
// when the levels need more shared memory than kSmallSmemLimit.
cudaError_t vcycle_small(const SmallVcycle& v, int nb, cudaStream_t s);

}  // namespace fmg
