// Fine-grid pass of the augmented nonlinear problem on the 3D Kuhn mesh: the per-coarse-
// tetrahedron integrals T3^T_abc = int_T u~ mu_a mu_b mu_c (the other moments, T0, T1 and
// the density stencil B(u~), come from grid3d.cu exactly as in 2D, see augment2d.cu).
//
// Coarse cell (I,J,L) holds 6 Kuhn tetrahedra T_s = {x_s0 >= x_s1 >= x_s2}; in the chain
// coordinates (a, b, c) = (x_s0, x_s1, x_s2) / r of a fine node (r fine cells per coarse
// cell) the barycentrics are mu = (1 - a, a - b, b - c, c) for every s, and the Kuhn mesh is
// symmetric under axis permutations, so one description serves all six.  T3 is linear in u~:
//   T3^T = sum_v u~_v int_T phi_v q,   q = mu_a mu_b mu_c (a cubic),
// and a Taylor expansion of q about node v is exact: int_T phi_v q = sum_{|b|<=3} D^b q(v)/b!
// m_b, m_b the moments of phi_v over the star tetrahedra of v inside T.  Those depend only
// on v's class - interior of T, one of 4 faces, 6 edges or 4 vertices - so T3 is a fixed
// linear map of the 15 x 20 class monomial sums S^class_g = sum u~ (a,b,c)^g, |g| <= 3.
#include <math.h>

#include <map>
#include <vector>

#include "fmg_internal.h"
#include "reduce_dev.cuh"

namespace fmg {
namespace {

constexpr int kThreads = 256;
constexpr int kMono = 20;       // monomials of degree <= 3 in 3 variables
constexpr int kClasses = 15;    // interior, F0..F3, E01 E02 E03 E12 E13 E23, V0..V3
constexpr int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
__constant__ int kPermDev[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// monomial order: degree 0; a b c; a^2 ab ac b^2 bc c^2; a^3 a^2b a^2c ab^2 abc ac^2 b^3 b^2c bc^2 c^3
__device__ __forceinline__ void monomials(double a, double b, double c, double* m) {
  m[0] = 1.0;
  m[1] = a; m[2] = b; m[3] = c;
  m[4] = a * a; m[5] = a * b; m[6] = a * c; m[7] = b * b; m[8] = b * c; m[9] = c * c;
  m[10] = m[4] * a; m[11] = m[4] * b; m[12] = m[4] * c; m[13] = a * m[7]; m[14] = m[5] * c;
  m[15] = a * m[9]; m[16] = m[7] * b; m[17] = m[7] * c; m[18] = b * m[9]; m[19] = m[9] * c;
}

// Interior class: a thread takes (x0, x2) lines of the coarse cell along x1 (kLinesPerThread of
// them, strided by the grid; x0 fastest across the threads: coalesced loads), block (chunk of
// lines, tet, instance), and adds their monomial sums before one block reduction (most of
// a line's FP64 work had been that reduction, many lines being empty).  On a line, the nodes
// strictly inside T_s are an interval of x1 (the chain order a > b > c of T_s bounds x1 by the
// line's two other coordinates), and every monomial is (powers of the line's fixed chain
// coordinates) x (a power of x1 / r): the thread sums u (x1/r)^e, e = 0..3, along its
// interval with the powers from the level's table pw (4 FMAs per node, in two interleaved
// sets of accumulators to halve the FP64 dependency chain) and then adds the 20 monomial
// sums of its line.
__constant__ int kMonoExpDev[20][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                       {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2},
                                       {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1},
                                       {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3}};

__device__ __forceinline__ int coord(int axis, int x0, int x1, int x2) {
  return axis == 0 ? x0 : (axis == 1 ? x1 : x2);
}

__device__ __forceinline__ double pick4(double v0, double v1, double v2, double v3, int e) {
  return e == 0 ? v0 : (e == 1 ? v1 : (e == 2 ? v2 : v3));
}

__global__ void __launch_bounds__(kThreads)
    k_t3_interior3d(int pf, long planef, int n1, int r, size_t st, size_t pst,
                    const double* __restrict__ u, const double* __restrict__ pw,
                    double* __restrict__ partials) {
  __shared__ double sh[kThreads];
  u += blockIdx.z * st;  // instance blockIdx.z
  partials += blockIdx.z * pst;
  const int tet = blockIdx.y;
  const int cell = tet / 6, s = tet % 6;
  const int I = cell % n1, J = (cell / n1) % n1, L = cell / (n1 * n1);
  const int R = r + 1;
  // chain position of axis 1 (the axis threads walk along)
  const int pos1 = kPermDev[s][0] == 1 ? 0 : (kPermDev[s][1] == 1 ? 1 : 2);
  double acc[kMono];
#pragma unroll
  for (int m = 0; m < kMono; ++m) acc[m] = 0.0;
  // a thread takes several lines (strided over the block's chunk of the grid) and sums their
  // monomial sums before the one block reduction
  for (int line = blockIdx.x * blockDim.x + threadIdx.x; line < R * R;
       line += gridDim.x * blockDim.x) {
    const int x0 = line % R, x2 = line / R;
    // the two fixed chain coordinates (positions q1 < q2, the ones other than pos1)
    const int q1 = pos1 == 0 ? 1 : 0, q2 = pos1 == 2 ? 1 : 2;
    const int f1 = coord(kPermDev[s][q1], x0, 0, x2), f2 = coord(kPermDev[s][q2], x0, 0, x2);
    // interval of x1 (exclusive bounds) from r > a > b > c > 0
    int lo = 0, hi = -1;
    if (pos1 == 0) {  // x1 = a, fixed b = f1, c = f2
      if (f1 > f2 && f2 > 0) { lo = f1; hi = r; }
    } else if (pos1 == 1) {  // x1 = b, fixed a = f1, c = f2
      if (f1 < r && f2 > 0) { lo = f2; hi = f1; }
    } else {  // x1 = c, fixed a = f1, b = f2
      if (f1 < r && f1 > f2) { lo = 0; hi = f2; }
    }
    if (lo + 1 < hi) {
      const double* colp =
          u + (size_t)(L * r + x2) * planef + (size_t)(J * r) * pf + (size_t)(I * r + x0);
      double m[2][4] = {{0.0, 0.0, 0.0, 0.0}, {0.0, 0.0, 0.0, 0.0}};
      int x1 = lo + 1;
      for (; x1 + 1 < hi; x1 += 2) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const double val = colp[(size_t)(x1 + h) * pf];
          const double* p = pw + 4 * (x1 + h);  // (x1/r)^e
          m[h][0] += val;
          m[h][1] = fma(val, p[1], m[h][1]);
          m[h][2] = fma(val, p[2], m[h][2]);
          m[h][3] = fma(val, p[3], m[h][3]);
        }
      }
      if (x1 < hi) {
        const double val = colp[(size_t)x1 * pf];
        const double* p = pw + 4 * x1;
        m[0][0] += val;
        m[0][1] = fma(val, p[1], m[0][1]);
        m[0][2] = fma(val, p[2], m[0][2]);
        m[0][3] = fma(val, p[3], m[0][3]);
      }
      const double m0 = m[0][0] + m[1][0], m1 = m[0][1] + m[1][1], m2 = m[0][2] + m[1][2],
                   m3 = m[0][3] + m[1][3];
      const double* g1p = pw + 4 * f1;
      const double* g2p = pw + 4 * f2;
#pragma unroll
      for (int q = 0; q < kMono; ++q) {
        const int e0 = kMonoExpDev[q][pos1], e1 = kMonoExpDev[q][q1], e2 = kMonoExpDev[q][q2];
        acc[q] = fma(g1p[e1] * g2p[e2], pick4(m0, m1, m2, m3, e0), acc[q]);
      }
    }
  }
  block_sum_to<kMono>(acc, sh, partials + ((size_t)tet * gridDim.x + blockIdx.x) * kMono);
}

// Boundary classes: block (class - 1, tet, instance).
//  * faces (F0..F3): two free chain coordinates p > q; a thread takes a row (fixed p) and
//    walks q, summing u (q/r)^e, e = 0..3, then adds the row's 20 monomial sums (each
//    monomial is a power of p/r times a power of q/r on a face);
//  * edges: one free coordinate, a thread per node; vertices: one node.
// Chain coordinates (a, b, c) of each class as functions of the free ones p > q > 0 (r fine
// cells per coarse cell): faces F0 (r, p, q), F1 (p, p, q), F2 (p, q, q), F3 (p, q, 0); edges
// E01 (r, r, p), E02 (r, p, p), E03 (r, p, 0), E12 (p, p, p), E13 (p, p, 0), E23 (p, 0, 0);
// vertices (0,0,0), (r,0,0), (r,r,0), (r,r,r).
__device__ __forceinline__ double pw3(double v, int e) {
  return e == 0 ? 1.0 : (e == 1 ? v : (e == 2 ? v * v : v * v * v));
}

__global__ void __launch_bounds__(kThreads)
    k_t3_boundary3d(int pf, long planef, int n1, int r, size_t st, size_t pst,
                    const double* __restrict__ u, double* __restrict__ partials) {
  __shared__ double sh[kThreads];
  u += blockIdx.z * st;  // instance blockIdx.z
  partials += blockIdx.z * pst;
  const int cls = 1 + blockIdx.x;
  const int tet = blockIdx.y;
  const int cell = tet / 6, s = tet % 6;
  const int I = cell % n1, J = (cell / n1) % n1, L = cell / (n1 * n1);
  const double inv_r = 1.0 / r;
  const double* base = u + (size_t)(L * r) * planef + (size_t)(J * r) * pf + (size_t)I * r;
  auto node = [&](int a, int b, int c) {
    int co[3];
    co[kPermDev[s][0]] = a;
    co[kPermDev[s][1]] = b;
    co[kPermDev[s][2]] = c;
    return base[(size_t)co[2] * planef + (size_t)co[1] * pf + co[0]];
  };
  double acc[kMono];
#pragma unroll
  for (int m = 0; m < kMono; ++m) acc[m] = 0.0;
  if (cls <= 4) {
    // face rows: p = 2 .. r - 1 (F0..F2) with q in (0, p), F0 with p < r; F3: a = p, b = q
    for (int p = 2 + threadIdx.x; p < r; p += blockDim.x) {
      double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
      for (int q = 1; q < p; ++q) {
        double v;
        switch (cls) {
          case 1: v = node(r, p, q); break;
          case 2: v = node(p, p, q); break;
          case 3: v = node(p, q, q); break;
          default: v = node(p, q, 0); break;
        }
        const double t = q * inv_r, t2 = t * t;
        m0 += v;
        m1 = fma(v, t, m1);
        m2 = fma(v, t2, m2);
        m3 = fma(v, t2 * t, m3);
      }
      const double g = p * inv_r;
#pragma unroll
      for (int k = 0; k < kMono; ++k) {
        const int ea = kMonoExpDev[k][0], eb = kMonoExpDev[k][1], ec = kMonoExpDev[k][2];
        int ep, eq;  // exponents of p / r and q / r of a^ea b^eb c^ec on the face
        bool zero = false;
        switch (cls) {
          case 1: ep = eb; eq = ec; break;           // (r, p, q)
          case 2: ep = ea + eb; eq = ec; break;      // (p, p, q)
          case 3: ep = ea; eq = eb + ec; break;      // (p, q, q)
          default: ep = ea; eq = eb; zero = ec > 0; break;  // (p, q, 0)
        }
        if (!zero && ep <= 3 && eq <= 3)
          acc[k] = fma(pw3(g, ep), pick4(m0, m1, m2, m3, eq), acc[k]);
      }
    }
  } else {
    // edges (one free coordinate p in (0, r)) and vertices (one node)
    const bool vertex = cls >= 11;
    for (int p = 1 + threadIdx.x; vertex ? (p == 1 && threadIdx.x == 0) : p < r;
         p += blockDim.x) {
      int abc[3];
      switch (cls) {
        case 5: abc[0] = r; abc[1] = r; abc[2] = p; break;   // E01
        case 6: abc[0] = r; abc[1] = p; abc[2] = p; break;   // E02
        case 7: abc[0] = r; abc[1] = p; abc[2] = 0; break;   // E03
        case 8: abc[0] = p; abc[1] = p; abc[2] = p; break;   // E12
        case 9: abc[0] = p; abc[1] = p; abc[2] = 0; break;   // E13
        case 10: abc[0] = p; abc[1] = 0; abc[2] = 0; break;  // E23
        case 11: abc[0] = 0; abc[1] = 0; abc[2] = 0; break;  // V0
        case 12: abc[0] = r; abc[1] = 0; abc[2] = 0; break;  // V1
        case 13: abc[0] = r; abc[1] = r; abc[2] = 0; break;  // V2
        default: abc[0] = r; abc[1] = r; abc[2] = r; break;  // V3
      }
      const double val = node(abc[0], abc[1], abc[2]);
      double m[kMono];
      monomials(abc[0] * inv_r, abc[1] * inv_r, abc[2] * inv_r, m);
#pragma unroll
      for (int k = 0; k < kMono; ++k) acc[k] = fma(val, m[k], acc[k]);
    }
  }
  block_sum_to<kMono>(acc, sh, partials + ((size_t)tet * (kClasses - 1) + blockIdx.x) * kMono);
}

// T3_e = h^3 sum_{class, g} map[e][class][g] S^class_g
__global__ void k_t3_finalize3d(int chunks, double h3, size_t pst, size_t tst,
                                const double* __restrict__ pin, const double* __restrict__ pbd,
                                const double* __restrict__ map, double* __restrict__ t3) {
  pin += blockIdx.y * pst;  // instance blockIdx.y
  pbd += blockIdx.y * pst;
  t3 += blockIdx.y * tst;
  const int tet = blockIdx.x;
  __shared__ double S[kClasses * kMono];
  for (int m = threadIdx.x; m < kMono; m += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < chunks; ++c) acc += pin[((size_t)tet * chunks + c) * kMono + m];
    S[m] = acc;
  }
  for (int e = threadIdx.x; e < (kClasses - 1) * kMono; e += blockDim.x)
    S[kMono + e] = pbd[(size_t)tet * (kClasses - 1) * kMono + e];
  __syncthreads();
  const int e = threadIdx.x;
  if (e >= 20) return;
  const double* row = map + (size_t)e * kClasses * kMono;
  double acc = 0.0;
  for (int q = 0; q < kClasses * kMono; ++q) acc = fma(row[q], S[q], acc);
  t3[(size_t)tet * 20 + e] = h3 * acc;
}

// Interior: a block takes interior_threads(r) lines (whole warps, up to kThreads) of the
// (r + 1)^2 lines of a tetrahedron.  Boundary: the face rows and edge nodes of a class number
// fewer than r, so a block of boundary_threads(r) covers them in one or a few passes.
int interior_threads(int r) { return warps_for((long)(r + 1) * (r + 1), kThreads); }
constexpr int kLinesPerThread = 8;  // lines summed per thread before the block reduction
int interior_chunks(int r) {
  const long rows = (long)(r + 1) * (r + 1);
  const long per_block = (long)interior_threads(r) * kLinesPerThread;
  return (int)((rows + per_block - 1) / per_block);
}
int boundary_threads(int r) { return warps_for(r, kThreads); }

// ---- host: class moments and the linear map ---------------------------------------------
// Polynomials in the 4 barycentrics of a tetrahedron, exponents packed in a key.
using Poly = std::map<int, double>;
int key(const int* e) { return e[0] | e[1] << 4 | e[2] << 8 | e[3] << 12; }
double fact(int k) {
  double r = 1.0;
  for (int i = 2; i <= k; ++i) r *= i;
  return r;
}
Poly mul(const Poly& x, const Poly& y) {
  Poly z;
  for (auto& a : x)
    for (auto& b : y) {
      int e[4];
      for (int i = 0; i < 4; ++i) e[i] = ((a.first >> (4 * i)) & 15) + ((b.first >> (4 * i)) & 15);
      z[key(e)] += a.second * b.second;
    }
  return z;
}
// int_K lambda^alpha for a tetrahedron of volume 1/6 (fine units): 6 |K| alpha! / (|alpha|+3)!
double integrate(const Poly& x) {
  double s = 0.0;
  for (auto& a : x) {
    int tot = 0;
    double num = 1.0;
    for (int i = 0; i < 4; ++i) {
      const int ei = (a.first >> (4 * i)) & 15;
      tot += ei;
      num *= fact(ei);
    }
    s += a.second * num / fact(tot + 3);
  }
  return s;
}

const int kMonoExp[20][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                             {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2},
                             {3, 0, 0}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {1, 1, 1},
                             {1, 0, 2}, {0, 3, 0}, {0, 2, 1}, {0, 1, 2}, {0, 0, 3}};

int mono_index(int a, int b, int c) {
  for (int q = 0; q < 20; ++q)
    if (kMonoExp[q][0] == a && kMonoExp[q][1] == b && kMonoExp[q][2] == c) return q;
  return -1;
}

// Moments m[class][g] = sum over the star tetrahedra of a class-representative node that lie
// in T = {R >= x0 >= x1 >= x2 >= 0} of int_K lambda_v (x - x_v)^g (fine units).
void class_moments3d(double mom[kClasses][kMono]) {
  const int R = 12;
  const int rep[kClasses][3] = {{9, 6, 3},   {12, 8, 4}, {8, 8, 4},  {8, 4, 4},   {8, 4, 0},
                                {12, 12, 6}, {12, 6, 6}, {12, 6, 0}, {6, 6, 6},   {6, 6, 0},
                                {6, 0, 0},   {0, 0, 0},  {12, 0, 0}, {12, 12, 0}, {12, 12, 12}};
  for (int cls = 0; cls < kClasses; ++cls) {
    for (int g = 0; g < kMono; ++g) mom[cls][g] = 0.0;
    const int* v = rep[cls];
    // the 8 cells around v and their Kuhn tetrahedra
    for (int o = 0; o < 8; ++o) {
      const int c0[3] = {v[0] - (o & 1), v[1] - ((o >> 1) & 1), v[2] - ((o >> 2) & 1)};
      for (int s = 0; s < 6; ++s) {
        int vt[4][3];
        for (int a = 0; a < 3; ++a) vt[0][a] = c0[a];
        for (int a = 0; a < 3; ++a) vt[1][a] = vt[0][a] + (a == kPerm[s][0]);
        for (int a = 0; a < 3; ++a) vt[2][a] = vt[1][a] + (a == kPerm[s][1]);
        for (int a = 0; a < 3; ++a) vt[3][a] = c0[a] + 1;
        int iv = -1;
        for (int w = 0; w < 4; ++w)
          if (vt[w][0] == v[0] && vt[w][1] == v[1] && vt[w][2] == v[2]) iv = w;
        if (iv < 0) continue;
        double cen[3] = {0, 0, 0};
        for (int w = 0; w < 4; ++w)
          for (int a = 0; a < 3; ++a) cen[a] += vt[w][a] / 4.0;
        if (!(R > cen[0] && cen[0] > cen[1] && cen[1] > cen[2] && cen[2] > 0)) continue;
        // x - x_v = sum_w lambda_w (x_w - x_v)
        Poly lin[3];
        for (int a = 0; a < 3; ++a)
          for (int w = 0; w < 4; ++w) {
            const double d = vt[w][a] - v[a];
            if (d == 0.0) continue;
            int e[4] = {0, 0, 0, 0};
            e[w] = 1;
            lin[a][key(e)] += d;
          }
        int ev[4] = {0, 0, 0, 0};
        ev[iv] = 1;
        for (int g = 0; g < kMono; ++g) {
          Poly p;
          p[key(ev)] = 1.0;
          for (int a = 0; a < 3; ++a)
            for (int k = 0; k < kMonoExp[g][a]; ++k) p = mul(p, lin[a]);
          mom[cls][g] += integrate(p);
        }
      }
    }
  }
}

// Every class sum is taken with the node's actual chain coordinates, so S^class_g is simply
// slot class * 20 + g.
void class_sum_terms(int cls, int ga, int gb, int gc, std::vector<std::pair<int, double>>& out) {
  out.clear();
  const int q = mono_index(ga, gb, gc);
  if (q >= 0) out.push_back({cls * kMono + q, 1.0});
}

}  // namespace

size_t t3_partials3d(const Grid& fine, int n1) {
  const int r = fine.n / n1;
  const size_t tets = (size_t)6 * n1 * n1 * n1;
  return tets * kMono * ((size_t)interior_chunks(r) + (kClasses - 1));
}

void t3_moments3d(const Grid& fine, int n1, const double* u, const double* pw,
                  const double* map, double* partials, double* t3, cudaStream_t s) {
  const int r = fine.n / n1;
  const int tets = 6 * n1 * n1 * n1;
  const int chunks = interior_chunks(r);
  const long planef = (long)(fine.n + 1) * fine.pitch;
  const size_t pst = t3_partials3d(fine, n1);  // per instance
  double* pin = partials;
  double* pbd = partials + (size_t)tets * chunks * kMono;
  k_t3_interior3d<<<dim3(chunks, tets, fine.nb), interior_threads(r), 0, s>>>(
      fine.pitch, planef, n1, r, fine.stride, pst, u, pw, pin);
  k_t3_boundary3d<<<dim3(kClasses - 1, tets, fine.nb), boundary_threads(r), 0, s>>>(
      fine.pitch, planef, n1, r, fine.stride, pst, u, pbd);
  k_t3_finalize3d<<<dim3(tets, fine.nb), 32, 0, s>>>(chunks, fine.h * fine.h * fine.h, pst,
                                                     (size_t)tets * 20, pin, pbd, map, t3);
}

// Host: map[e][class][g] for T3_e = h^3 sum map S^class_g (r fine cells per coarse cell),
//   T3_e = sum_class sum_{|b|<=3} m^class_b r^-|b| / b! sum_{|g|<=3} c^e_g (g)_b S^class_{g-b},
// c^e the monomial coefficients of q_e = mu_a mu_b mu_c in chain coordinates and (g)_b the
// falling factorials.
void t3_map3d(int r, double* out) {
  double mom[kClasses][kMono];
  class_moments3d(mom);
  for (int i = 0; i < 20 * kClasses * kMono; ++i) out[i] = 0.0;
  // barycentrics (const, a, b, c) coefficients
  const double mu[4][4] = {{1, -1, 0, 0}, {0, 1, -1, 0}, {0, 0, 1, -1}, {0, 0, 0, 1}};
  auto ff = [](int g, int b) {  // falling factorial (g)_b
    double r = 1.0;
    for (int i = 0; i < b; ++i) r *= (g - i);
    return r;
  };
  std::vector<std::pair<int, double>> terms;
  int e = 0;
  for (int x = 0; x < 4; ++x)
    for (int y = x; y < 4; ++y)
      for (int z = y; z < 4; ++z, ++e) {
        double cq[4][4][4] = {};
        cq[0][0][0] = 1.0;
        const int f3[3] = {x, y, z};
        for (int f = 0; f < 3; ++f) {
          double nq[4][4][4] = {};
          const double* m = mu[f3[f]];
          for (int a = 0; a < 4; ++a)
            for (int b = 0; a + b < 4; ++b)
              for (int c = 0; a + b + c < 4; ++c) {
                if (cq[a][b][c] == 0.0) continue;
                nq[a][b][c] += cq[a][b][c] * m[0];
                if (a + b + c + 1 < 4) {
                  nq[a + 1][b][c] += cq[a][b][c] * m[1];
                  nq[a][b + 1][c] += cq[a][b][c] * m[2];
                  nq[a][b][c + 1] += cq[a][b][c] * m[3];
                }
              }
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
              for (int c = 0; c < 4; ++c) cq[a][b][c] = nq[a][b][c];
        }
        double* row = out + (size_t)e * kClasses * kMono;
        for (int cls = 0; cls < kClasses; ++cls)
          for (int bq = 0; bq < kMono; ++bq) {
            const double mb = mom[cls][bq];
            if (mb == 0.0) continue;
            const int b0 = kMonoExp[bq][0], b1 = kMonoExp[bq][1], b2 = kMonoExp[bq][2];
            const double w = mb * pow((double)r, -(b0 + b1 + b2)) / (fact(b0) * fact(b1) * fact(b2));
            for (int g0 = b0; g0 < 4; ++g0)
              for (int g1 = b1; g0 + g1 < 4; ++g1)
                for (int g2 = b2; g0 + g1 + g2 < 4; ++g2) {
                  const double cg = cq[g0][g1][g2];
                  if (cg == 0.0) continue;
                  const double coef = w * cg * ff(g0, b0) * ff(g1, b1) * ff(g2, b2);
                  class_sum_terms(cls, g0 - b0, g1 - b1, g2 - b2, terms);
                  for (auto& t : terms) row[t.first] += coef * t.second;
                }
          }
      }
}

}  // namespace fmg
