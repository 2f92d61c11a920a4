// Moments of u~ that make the nonlinear term of the augmented problem (Algorithm 3.1 step 2)
// an O(#coarse elements) computation per nonlinear iteration.
//
// On the augmented space V_H + span{u~} every w = w_H + c_u u~, and the nonlinear matrix
// G(c)_ij = int w^2 psi_i psi_j expands into integrals of u~^p times products of coarse
// barycentric coordinates mu_a (linear on each coarse triangle T):
//   int_T u~^4, int_T u~^3 mu_a, int_T u~^2 mu_a mu_b, int_T u~ mu_a mu_b mu_c.
// One pass over the fine triangles per correction step computes all of them; the small
// nonlinear solve then never touches the fine grid again (the paper assembles the augmented
// matrix with an O(N_k) pass per nonlinear iteration, Section 3.2).
//
// Every integrand is a polynomial of degree 4 on a fine triangle, integrated exactly by a
// symmetric 6-point rule of degree 4 whose parameters the host solves from its moment
// equations.  Fine triangle (a,b) of a coarse cell lies in coarse triangle 0 = (V00,V10,V11)
// (the part s >= t) or 1 = (V00,V11,V01).  Reductions are fixed-order block trees followed by
// a fixed-order sum over chunks, so results are deterministic.
#include "fmg_internal.h"

namespace fmg {
namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 8;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;

struct Rule {
  double a1, b1, w1, a2, b2, w2;  // orbits (a, b, b); weights per point (area factor folded)
};

template <int T>
__device__ __forceinline__ void accumulate_point(double s, double t, double inv_r, double u,
                                                 double w, double* acc) {
  const double sg = s * inv_r, tg = t * inv_r;
  double m0, m1, m2;
  if (T == 0) {
    m0 = 1.0 - sg;
    m1 = sg - tg;
    m2 = tg;
  } else {
    m0 = 1.0 - tg;
    m1 = sg;
    m2 = tg - sg;
  }
  const double wu = w * u, wu2 = wu * u, wu3 = wu2 * u;
  acc[0] = fma(wu3, u, acc[0]);
  acc[1] = fma(wu3, m0, acc[1]);
  acc[2] = fma(wu3, m1, acc[2]);
  acc[3] = fma(wu3, m2, acc[3]);
  const double q00 = m0 * m0, q01 = m0 * m1, q02 = m0 * m2, q11 = m1 * m1, q12 = m1 * m2,
               q22 = m2 * m2;
  acc[4] = fma(wu2, q00, acc[4]);
  acc[5] = fma(wu2, q01, acc[5]);
  acc[6] = fma(wu2, q02, acc[6]);
  acc[7] = fma(wu2, q11, acc[7]);
  acc[8] = fma(wu2, q12, acc[8]);
  acc[9] = fma(wu2, q22, acc[9]);
  acc[10] = fma(wu * q00, m0, acc[10]);
  acc[11] = fma(wu * q00, m1, acc[11]);
  acc[12] = fma(wu * q00, m2, acc[12]);
  acc[13] = fma(wu * q01, m1, acc[13]);
  acc[14] = fma(wu * q01, m2, acc[14]);
  acc[15] = fma(wu * q02, m2, acc[15]);
  acc[16] = fma(wu * q11, m1, acc[16]);
  acc[17] = fma(wu * q11, m2, acc[17]);
  acc[18] = fma(wu * q12, m2, acc[18]);
  acc[19] = fma(wu * q22, m2, acc[19]);
}

// One fine triangle with vertex positions (s_v, t_v) in fine-cell units from the coarse
// cell's corner and vertex values u_v.
template <int T>
__device__ __forceinline__ void accumulate_triangle(const double* s, const double* t,
                                                    const double* u, double inv_r,
                                                    const Rule& q, double* acc) {
  const double ss = s[0] + s[1] + s[2], ts = t[0] + t[1] + t[2], us = u[0] + u[1] + u[2];
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    const double a = o == 0 ? q.a1 : q.a2;
    const double b = o == 0 ? q.b1 : q.b2;
    const double w = o == 0 ? q.w1 : q.w2;
    const double d = a - b;
    const double bs = b * ss, bt = b * ts, bu = b * us;
#pragma unroll
    for (int v = 0; v < 3; ++v)
      accumulate_point<T>(fma(d, s[v], bs), fma(d, t[v], bt), inv_r, fma(d, u[v], bu), w, acc);
  }
}

__device__ void block_reduce_store(double* acc, double* sh, double* out) {
  for (int m = 0; m < kMom; ++m) {
    sh[threadIdx.x] = acc[m];
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[m] = sh[0];
    __syncthreads();
  }
}

// grid: x = chunk of fine cells, y = coarse triangle (2 * cell + T)
template <int T>
__device__ void moments_body(int pf, int n1, int r, const double* __restrict__ u,
                             double* __restrict__ partials, Rule q) {
  __shared__ double sh[kThreads];
  const int tri = blockIdx.y;
  const int cell = tri >> 1;
  const int I = cell % n1, J = cell / n1;
  const size_t cells = (size_t)r * r;
  const size_t beg = (size_t)blockIdx.x * kCellsPerBlock;
  const double inv_r = 1.0 / r;
  double acc[kMom];
#pragma unroll
  for (int m = 0; m < kMom; ++m) acc[m] = 0.0;
  for (int it = 0; it < kCellsPerThread; ++it) {
    const size_t idx = beg + (size_t)it * kThreads + threadIdx.x;
    if (idx >= cells) break;
    const int a = (int)(idx % r), b = (int)(idx / r);
    // fine triangle 1 (V00,V10,V11) lies in coarse triangle 0 iff a >= b;
    // fine triangle 2 (V00,V11,V01) lies in coarse triangle 0 iff a > b.
    const bool use1 = T == 0 ? (a >= b) : (a < b);
    const bool use2 = T == 0 ? (a > b) : (a <= b);
    if (!use1 && !use2) continue;
    const size_t k = (size_t)(J * r + b) * pf + (size_t)(I * r + a);
    const double u00 = u[k], u10 = u[k + 1], u11 = u[k + pf + 1], u01 = u[k + pf];
    const double da = a, db = b;
    if (use1) {
      const double s[3] = {da, da + 1.0, da + 1.0}, t[3] = {db, db, db + 1.0};
      const double uv[3] = {u00, u10, u11};
      accumulate_triangle<T>(s, t, uv, inv_r, q, acc);
    }
    if (use2) {
      const double s[3] = {da, da + 1.0, da}, t[3] = {db, db + 1.0, db + 1.0};
      const double uv[3] = {u00, u11, u01};
      accumulate_triangle<T>(s, t, uv, inv_r, q, acc);
    }
  }
  block_reduce_store(acc, sh, partials + ((size_t)tri * gridDim.x + blockIdx.x) * kMom);
}

__global__ void __launch_bounds__(kThreads) k_moments2d(int pf, int n1, int r,
                                                        const double* __restrict__ u,
                                                        double* __restrict__ partials, Rule q) {
  if (blockIdx.y & 1)
    moments_body<1>(pf, n1, r, u, partials, q);
  else
    moments_body<0>(pf, n1, r, u, partials, q);
}

__global__ void k_moments_final(int chunks, const double* __restrict__ partials,
                                double* __restrict__ out) {
  const int tri = blockIdx.x;
  const int m = threadIdx.x;
  if (m >= kMom) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += partials[((size_t)tri * chunks + c) * kMom + m];
  out[(size_t)tri * kMom + m] = s;
}

int chunks_for(int r) {
  const size_t cells = (size_t)r * r;
  return (int)((cells + kCellsPerBlock - 1) / kCellsPerBlock);
}

}  // namespace

size_t moments2d_partials(const Grid& fine, int n1) {
  const int r = fine.n / n1;
  return (size_t)2 * n1 * n1 * chunks_for(r) * kMom;
}

void moments2d(const Grid& fine, int n1, const double* u, double* partials, double* out,
               const double rule[4], cudaStream_t s) {
  const int r = fine.n / n1;
  const int chunks = chunks_for(r);
  const double area = fine.h * fine.h / 2.0;
  Rule q;
  q.a1 = rule[0];
  q.b1 = 0.5 * (1.0 - rule[0]);
  q.w1 = rule[1] / 3.0 * area;
  q.a2 = rule[2];
  q.b2 = 0.5 * (1.0 - rule[2]);
  q.w2 = rule[3] / 3.0 * area;
  dim3 grid(chunks, 2 * n1 * n1);
  k_moments2d<<<grid, kThreads, 0, s>>>(fine.pitch, n1, r, u, partials, q);
  k_moments_final<<<2 * n1 * n1, 32, 0, s>>>(chunks, partials, out);
}

}  // namespace fmg
