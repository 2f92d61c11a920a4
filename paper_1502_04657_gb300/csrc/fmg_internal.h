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

struct Grid {
  int dim = 2;
  int n = 0;          // cells per side
  int pitch = 0;      // elements per row
  int rows = 0;       // rows per plane (n + 1)
  size_t stride = 0;  // elements per vector
  double h = 0;
  size_t interior() const {
    size_t m = (size_t)(n - 1);
    return dim == 2 ? m * m : m * m * m;
  }
};

// Stencil coefficients of L = A + W on one 2D level (see grid2d.cu for the closed forms).
struct Coef2D {
  double* cC;    // diagonal
  double* cE;    // coupling (i,j)-(i+1,j)
  double* cN;    // coupling (i,j)-(i,j+1)
  double* cNE;   // coupling (i,j)-(i+1,j+1)
  double* dinv;  // omega / cC
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
void jacobi2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* xo,
              bool x_is_zero, cudaStream_t s);
void residual2d(const Grid& g, const Coef2D& c, const double* f, const double* x, double* r,
                cudaStream_t s);
void restrict2d(const Grid& fine, const Grid& coarse, const double* rf, double* rc,
                cudaStream_t s);
// xf = (add ? xf : 0) + P ec (+ scale[0] * extra when extra != nullptr)
void prolong2d(const Grid& fine, const Grid& coarse, const double* ec, double* xf, bool add,
               const double* extra, const double* scale, cudaStream_t s);
void nload2d(const Grid& g, const double* u, double* out, cudaStream_t s);
// f = lam[0] * M u - p->zeta * N(u)
void rhs2d(const Grid& g, const double* lam, const PotentialParams* p_dev, const double* u,
           double* f, cudaStream_t s);
// Dense level-1 matrices L_1 and M_1 (n1-1)^2 square, row-major, interior numbering.
void dense_level1_2d(const Grid& g, const Coef2D& c, double* L, double* M, cudaStream_t s);
// sin-product start vector for the level-1 nonlinear solve
void start_vector(const Grid& g, double box_len, double* c, cudaStream_t s);

// ---- Reductions (reduce.cu) -------------------------------------------------------------
// out[0] = sum_i a[i] * b[i] over n entries; deterministic two-stage tree.  `partials` holds
// at least kReduceBlocks doubles.
constexpr int kReduceBlocks = 1024;
void dot(const double* a, const double* b, size_t n, double* partials, double* out,
         cudaStream_t s);

// ---- Interior <-> padded packing (pack.cu) ----------------------------------------------
void pack_interior(const Grid& g, const double* interior, double* padded, cudaStream_t s);
void unpack_interior(const Grid& g, const double* padded, double* interior, cudaStream_t s);
// padded level-1 vector from a dense coefficient vector c (first n1 entries)
void scatter_level1(const Grid& g, const double* c, double* padded, cudaStream_t s);

// ---- Augmented-space moments (moments2d.cu) ----------------------------------------------
// Per coarse triangle (2 per coarse cell, coarse cell index = I + n1 * J, triangle
// 2 * cell + {0: (V00,V10,V11), 1: (V00,V11,V01)}): 20 moments of u~ against the coarse
// barycentric coordinates mu_a of that triangle:
//   [0] int u^4, [1..3] int u^3 mu_a, [4..9] int u^2 mu_a mu_b (a<=b: 00,01,02,11,12,22),
//   [10..19] int u mu_a mu_b mu_c (a<=b<=c: 000,001,002,011,012,022,111,112,122,222).
constexpr int kMom = 20;
size_t moments2d_partials(const Grid& fine, int n1);  // doubles of scratch needed
void moments2d(const Grid& fine, int n1, const double* u, double* partials, double* out,
               const double rule[4], cudaStream_t s);

// ---- Dense small solves (dense.cu) -------------------------------------------------------
struct DenseProblem {
  int nh;              // coarse unknowns (interior nodes of level 1)
  int aug;             // 1: basis (phi^H, u~), n = nh + 1; 0: basis phi^H, n = nh
  int ntri;            // coarse simplices
  int nvert;           // vertices per simplex (3 in 2D, 4 in 3D)
  const int* tri;      // ntri * nvert coarse interior indices, -1 on the boundary
  const int* adj;      // nh * maxadj codes (simplex << 3 | local vertex), -1 terminated
  int maxadj;
  const double* q4;    // nvert^4 table: int_T mu_a mu_b mu_c mu_d / |T|
  double tri_vol;      // |T|
  const double* L1;    // nh*nh
  const double* M1;    // nh*nh
  const double* gA;    // padded level-1 vector P^T..P^T L u~        (aug)
  const double* gM;    // padded level-1 vector P^T..P^T M u~        (aug)
  const double* auu;   // u~^T L u~                                    (aug)
  const double* buu;   // u~^T M u~                                    (aug)
  const double* mom;   // ntri * kMom (2D) moments                     (aug)
  int n1;              // cells per side of level 1 (to read padded gA/gM)
  int pitch1;
  const PotentialParams* params;  // device; zeta read from here
  double tol;
  int max_iter;
  const double* c_init;  // nullptr: augmented start e_u / sqrt(buu); level-1: caller fills
  double* c_out;         // n
  double* lam_out;       // 1
  int* iters_out;        // 1
  int* status_out;       // 1 (0 converged, 1 cap hit)
};
constexpr size_t kDenseSmemLimit = 200 * 1024;  // dynamic shared memory of the dense solve
size_t dense_smem_bytes(int n, int ntri, int nvert);
cudaError_t dense_prepare(size_t max_smem);  // opt in to large dynamic shared memory
void dense_scf(const DenseProblem& p, cudaStream_t s);
// Linv = L^{-1} for an SPD n x n matrix (Cholesky), one CTA.
void dense_spd_inverse(const double* L, double* Linv, int n, cudaStream_t s);
// y(padded level 1) = Linv * x(padded level 1) on the interior nodes
void coarse_matvec2d(const Grid& g, const double* Linv, const double* x, double* y,
                     cudaStream_t s);

}  // namespace fmg
