// CPU oracle for the decomposed ("parallel") sequential sweep of
// R. Tavakoli, "Parallelizing sequential sweeping on structured grids --
// fully parallel SOR/ILU preconditioners for structured n-diagonal matrices"
// (arXiv 1008.3699).
//
// TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library. The product
// path (the CUDA library under paper_1008_3699_gb300/) never calls it, shares no
// code, header, table or constant with it, and fails loudly when its own
// extension is missing.
//
// Plain, slow, obviously-correct single-threaded C++ in fp64 (built with
// -ffp-contract=off, no fast-math). Every function states the passage of the
// paper it follows:
//
//   matrix / stencil layout .......... Eq. (d2d), Sec. 3; Def. "structured
//                                      n-diagonal matrix", Sec. 7
//   Cartesian partition ............... Sec. 3, "Domain decomposition"
//   sweep-direction schedule .......... Sec. 2 steps (ii)/(iii) for 1D,
//                                      Sec. 3 "Sweeping directions", Sec. 4 (3D)
//   implicit set J_i of a sweep ....... Eqs. (sor2d_sw..nw), (2d:sor4b4),
//                                      (2d:sor2b2); the splitting form of one
//                                      parallel iteration, Eq. (ca2d:matiter)
//   coupled systems ................... strongly connected components of the
//                                      implicit-dependency graph, solved
//                                      exactly (Eqs. 1d:sorc, 2d:sor4b4,
//                                      2d:sor2b2; Sec. 4: 8x8/4x4/2x2 in 3D)
//   ILU(0) ............................ Sec. 5 (SGS pass == ILU(0), Saad 10.3)
//   decomposed full ILU(0) ............ Sec. 5 read per subdomain block: the
//                                      IKJ elimination (Saad Alg. 10.4) of
//                                      A's block in its sweep order, couplings
//                                      across interfaces those of the sweep
//   SSOR apply (SPD form) ............. Sec. 2 (SSOR = LR then RL), Sec. 5
//   Krylov drivers .................... standard PCG / right-preconditioned
//                                      BiCGSTAB (not from the paper)
//   fast sweeping (eikonal) ........... closing remarks of the paper (the
//                                      same decomposition for the fast
//                                      sweeping method); Zhao's Godunov update
//
// Pins (tests/test_oracle_*.py): Table 1 iteration counts (1D GS natural and
// decomposed), closed-form SOR/GS contraction rates on the Poisson model,
// dense direct solves, the splitting equation, (LU)_ij = A_ij on the ILU(0)
// pattern, SSOR symmetry and its dense closed form; the full ILU(0): natural
// IKJ with one subdomain, (LU)_ij = A_ij on every block's pattern, the
// textbook ILU(1) of every block for 5-point matrices in 9-point storage, and
// the apply against the dense product of its factors.
// "parity unpinned" for the decomposed sweep and ILU on the 9-point stencil,
// as a reading: Sec. 3 gives no detail, so which diagonal neighbours are new
// is a choice. The code is checked against that reading by computations
// outside it: the face implicit sets equal the 5-point ones (pinned to the
// printed systems), a 5-point matrix in 9-point storage sweeps as the 5-point
// problem, and with cross-interface face couplings removed each subdomain is
// natural SOR of its reflected block (dense solve). The 9-point D-ILU pivots
// are pinned by D-ILU's definition, diag(M) = diag(A).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <utility>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Grid and stencil (Eq. d2d; Def. of a structured n-diagonal matrix, Sec. 7).
// Entry k of a row is A(i, i + off_k). Order of the entries:
//   3-pt (1D): C W E
//   5-pt (2D): C W E S N
//   7-pt (3D): C W E S N B F
//   9-pt (2D): C W E S N SW SE NW NE
// Cells are numbered naturally, x fastest (Sec. 3, "Data structure").
// Entries that point outside the grid are ignored (Dirichlet values are
// folded into the right-hand side, Eq. 1d:mat).
// ---------------------------------------------------------------------------
struct Grid {
  int d = 0;
  int64_t n[3] = {1, 1, 1};
  int s = 0;
  int off[9][3] = {};
  int opp[9] = {};
  int64_t N = 0;
};

bool make_grid(Grid& g, int d, const int64_t* n, int s) {
  if (d < 1 || d > 3) return false;
  g.d = d;
  for (int a = 0; a < 3; ++a) g.n[a] = (a < d) ? n[a] : 1;
  for (int a = 0; a < d; ++a)
    if (g.n[a] < 1) return false;
  g.s = s;
  static const int o3[3][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}};
  static const int o5[5][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}};
  static const int o7[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                               {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  static const int o9[9][3] = {{0, 0, 0},  {-1, 0, 0}, {1, 0, 0},  {0, -1, 0}, {0, 1, 0},
                               {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0}};
  const int(*o)[3] = nullptr;
  if (d == 1 && s == 3) o = o3;
  else if (d == 2 && s == 5) o = o5;
  else if (d == 3 && s == 7) o = o7;
  else if (d == 2 && s == 9) o = o9;
  else return false;
  for (int k = 0; k < s; ++k)
    for (int a = 0; a < 3; ++a) g.off[k][a] = o[k][a];
  for (int k = 0; k < s; ++k)
    for (int m = 0; m < s; ++m)
      if (o[m][0] == -o[k][0] && o[m][1] == -o[k][1] && o[m][2] == -o[k][2]) g.opp[k] = m;
  g.N = g.n[0] * g.n[1] * g.n[2];
  return true;
}

inline void coords(const Grid& g, int64_t i, int64_t c[3]) {
  c[0] = i % g.n[0];
  c[1] = (i / g.n[0]) % g.n[1];
  c[2] = i / (g.n[0] * g.n[1]);
}

// Neighbour of cell i along stencil entry k, or -1 outside the grid.
inline int64_t neighbour(const Grid& g, int64_t i, int k) {
  int64_t c[3];
  coords(g, i, c);
  for (int a = 0; a < 3; ++a) {
    c[a] += g.off[k][a];
    if (c[a] < 0 || c[a] >= g.n[a]) return -1;
  }
  return c[0] + g.n[0] * (c[1] + g.n[1] * c[2]);
}

// ---------------------------------------------------------------------------
// Cartesian partition into p_x x p_y x p_z nearly equal subdomains
// (Sec. 3, "Domain decomposition"): n cells into p parts, the first n mod p
// parts get one extra cell.
// ---------------------------------------------------------------------------
struct Partition {
  int p[3] = {1, 1, 1};
  std::vector<int64_t> lo[3];      // lo[a][q] = first coordinate of part q
  std::vector<int> part_of[3];     // part_of[a][x] = part index of coordinate x
};

bool make_partition(const Grid& g, const int* sub, Partition& P) {
  for (int a = 0; a < 3; ++a) {
    int p = (a < g.d) ? sub[a] : 1;
    if (p < 1 || p > g.n[a]) return false;
    P.p[a] = p;
    P.lo[a].assign(p + 1, 0);
    int64_t q = g.n[a] / p, r = g.n[a] % p;
    for (int k = 0; k < p; ++k) P.lo[a][k + 1] = P.lo[a][k] + q + (k < r ? 1 : 0);
    P.part_of[a].assign(g.n[a], 0);
    for (int k = 0; k < p; ++k)
      for (int64_t x = P.lo[a][k]; x < P.lo[a][k + 1]; ++x) P.part_of[a][x] = k;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Sweep-direction schedule. A direction is the start corner c, bit a set when
// the subdomain starts at its maximum coordinate along axis a (sweeps -a).
//
// 1D (Sec. 2, steps (ii)-(iii)): odd and even subdomains sweep in opposite
//   directions and every direction reverses after each iteration; the first
//   subdomain sweeps left-to-right at the first iteration.
// 2D (Sec. 3, the 2x2 example; "Sweeping directions"): subdomain (0,0) sweeps NE->SW,
//   then SW->NE, then NW->SE, then SE->NW (four-iteration cycle); a neighbour
//   along axis a has bit a flipped.
// 3D (Sec. 4: the 2D rules with eight directions; the order is not given):
//   within each pair of sweeps the direction is reversed, and pair g starts
//   from the all-ones corner with g's two bits flipped on axes x and y.
// ---------------------------------------------------------------------------
int base_corner(int d, int64_t t) {
  if (d == 1) return (int)(t & 1);
  const int period = 1 << d;
  const int tt = (int)(((t % period) + period) % period);
  const int all = period - 1;
  int c = all ^ (tt >> 1);
  if (tt & 1) c = all ^ c;
  return c;
}

int subdomain_corner(int d, int64_t t, const int idx[3]) {
  int c = base_corner(d, t);
  for (int a = 0; a < d; ++a)
    if (idx[a] & 1) c ^= (1 << a);
  return c;
}

// ---------------------------------------------------------------------------
// Problem handle.
// ---------------------------------------------------------------------------
enum { MODE_NATURAL = 0, MODE_DECOMPOSED = 1, MODE_DECOMPOSED_FULL = 3 };

struct Plan {
  bool built = false;
  std::vector<uint16_t> jmask;   // bit k: neighbour along entry k is in J_i
  std::vector<int64_t> order;    // cells, grouped by coupled block, in solve order
  std::vector<int64_t> bstart;   // block b = order[bstart[b] .. bstart[b+1])
  std::vector<uint8_t> corner;   // start corner of the cell's subdomain
};

struct Problem {
  Grid g;
  Partition P;
  std::vector<double> A;         // s x N, diagonal-major
  Plan plans[2][8];              // [mode][t mod 2^d]
  // ILU(0)
  int ilu_mode = -1;
  std::vector<double> dtilde;    // decomposed ILU(0) pivots
  std::vector<double> lu;        // natural ILU(0): s x N, L multipliers / U
  std::vector<double> full;      // decomposed full ILU(0): s x N in the form (D + L') D^-1 (D + U')
  // per-iteration record of the last Krylov solve, 4 values per iteration:
  // BiCGSTAB ||s||/||b||, ||r||/||b||, alpha, omega; PCG ||r||/||b||, alpha, 0, 0
  std::vector<double> hist;
};

inline double aval(const Problem& pb, int k, int64_t i) { return pb.A[(size_t)k * pb.g.N + i]; }

int cell_corner(const Problem& pb, int64_t t, const int64_t c[3]) {
  int idx[3];
  for (int a = 0; a < 3; ++a) idx[a] = pb.P.part_of[a][c[a]];
  return subdomain_corner(pb.g.d, t, idx);
}

bool same_part(const Problem& pb, const int64_t a[3], const int64_t b[3]) {
  for (int ax = 0; ax < 3; ++ax)
    if (pb.P.part_of[ax][a[ax]] != pb.P.part_of[ax][b[ax]]) return false;
  return true;
}

// Order key of a cell inside a subdomain with start corner cs: coordinates
// reflected along every axis the subdomain sweeps backwards; cells are visited
// in lexicographic order of (z, y, x) of the reflected coordinates. For the
// 5/7-point molecules this is any of the orders of Fig. swp2d (row-wise or
// frontal) -- they give the same iterate because the face neighbours that are
// already new are exactly the upstream ones (Eqs. sor2d_sw..nw).
bool precedes(const int64_t q[3], const int64_t i[3], int cs) {
  for (int a = 2; a >= 0; --a) {
    int64_t kq = (cs >> a & 1) ? -q[a] : q[a];
    int64_t ki = (cs >> a & 1) ? -i[a] : i[a];
    if (kq != ki) return kq < ki;
  }
  return false;
}

// Implicit set J_i of one sweep (the "new values" in Eqs. sor2d_sw..nw and the
// unknowns of the coupled systems (2d:sor4b4), (2d:sor2b2)):
//  natural mode:    neighbours with a lower natural index;
//  decomposed mode: (a) neighbours in the same subdomain that precede i in its
//                   sweep order, and (b) face neighbours in another subdomain
//                   that are upstream of i in i's sweep while i is upstream of
//                   them in theirs (both subdomains start at the shared
//                   interface, so the pair is solved together). Every other
//                   neighbour keeps its old value (halo semantics, Sec. 3,
//                   "Data structure").
bool implicit(const Problem& pb, int mode, int64_t t, int64_t i, int k, int64_t q) {
  if (mode == MODE_NATURAL) return q < i;
  int64_t ci[3], cq[3];
  coords(pb.g, i, ci);
  coords(pb.g, q, cq);
  const int csi = cell_corner(pb, t, ci);
  if (same_part(pb, ci, cq)) return precedes(cq, ci, csi);
  int axis = -1, nz = 0;
  for (int a = 0; a < 3; ++a)
    if (pb.g.off[k][a] != 0) { axis = a; ++nz; }
  if (nz != 1) return false;  // diagonal neighbour across an interface: old value
  const int csq = cell_corner(pb, t, cq);
  const bool q_up_in_i = (csi >> axis & 1) ? (cq[axis] > ci[axis]) : (cq[axis] < ci[axis]);
  const bool i_up_in_q = (csq >> axis & 1) ? (ci[axis] > cq[axis]) : (ci[axis] < cq[axis]);
  return q_up_in_i && i_up_in_q;
}

// Strongly connected components of the graph i -> j (j in J_i), by Tarjan's
// algorithm (iterative). Tarjan emits a component only after every component
// it can reach, i.e. after all of its dependencies, so the emission order is a
// valid solve order. A component with more than one cell is a coupled system
// of the paper (the 2x2 systems of Eq. 1d:sorc / 2d:sor2b2, the 4x4 corner
// system of Eq. 2d:sor4b4, the 8x8/4x4/2x2 systems of Sec. 4).
void build_plan(Problem& pb, int mode, int64_t t, Plan& pl) {
  const Grid& g = pb.g;
  const int64_t N = g.N;
  pl.jmask.assign(N, 0);
  pl.corner.assign(N, 0);
  for (int64_t i = 0; i < N; ++i) {
    int64_t c[3];
    coords(g, i, c);
    pl.corner[i] = (uint8_t)(mode == MODE_NATURAL ? 0 : cell_corner(pb, t, c));
    for (int k = 1; k < g.s; ++k) {
      int64_t q = neighbour(g, i, k);
      if (q >= 0 && implicit(pb, mode, t, i, k, q)) pl.jmask[i] |= (uint16_t)(1u << k);
    }
  }
  std::vector<int64_t> index(N, -1), low(N, 0);
  std::vector<uint8_t> onstack(N, 0);
  std::vector<int64_t> stack;
  struct Frame { int64_t v; int k; };
  std::vector<Frame> call;
  pl.order.clear();
  pl.bstart.assign(1, 0);
  int64_t counter = 0;
  for (int64_t root = 0; root < N; ++root) {
    if (index[root] >= 0) continue;
    call.push_back({root, 1});
    index[root] = low[root] = counter++;
    stack.push_back(root);
    onstack[root] = 1;
    while (!call.empty()) {
      Frame& f = call.back();
      const int64_t v = f.v;
      bool descended = false;
      while (f.k < g.s) {
        const int k = f.k++;
        if (!(pl.jmask[v] >> k & 1)) continue;
        const int64_t w = neighbour(g, v, k);
        if (index[w] < 0) {
          index[w] = low[w] = counter++;
          stack.push_back(w);
          onstack[w] = 1;
          call.push_back({w, 1});
          descended = true;
          break;
        } else if (onstack[w]) {
          if (index[w] < low[v]) low[v] = index[w];
        }
      }
      if (descended) continue;
      if (low[v] == index[v]) {
        int64_t w;
        do {
          w = stack.back();
          stack.pop_back();
          onstack[w] = 0;
          pl.order.push_back(w);
        } while (w != v);
        pl.bstart.push_back((int64_t)pl.order.size());
      }
      call.pop_back();
      if (!call.empty()) {
        const int64_t u = call.back().v;
        if (low[v] < low[u]) low[u] = low[v];
      }
    }
  }
  pl.built = true;
}

Plan& get_plan(Problem& pb, int mode, int64_t t) {
  const int period = 1 << pb.g.d;
  const int tt = (mode == MODE_NATURAL) ? 0 : (int)(((t % period) + period) % period);
  Plan& pl = pb.plans[mode][tt];
  if (!pl.built) build_plan(pb, mode, tt, pl);
  return pl;
}

// Dense Gaussian elimination with partial pivoting, m x m (row-major).
bool dense_solve(int m, std::vector<double>& M, std::vector<double>& r, std::vector<double>& x) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int rr = c + 1; rr < m; ++rr)
      if (std::fabs(M[rr * m + c]) > std::fabs(M[piv * m + c])) piv = rr;
    if (M[piv * m + c] == 0.0) return false;
    if (piv != c) {
      for (int cc = 0; cc < m; ++cc) std::swap(M[c * m + cc], M[piv * m + cc]);
      std::swap(r[c], r[piv]);
    }
    for (int rr = c + 1; rr < m; ++rr) {
      const double f = M[rr * m + c] / M[c * m + c];
      if (f == 0.0) continue;
      for (int cc = c; cc < m; ++cc) M[rr * m + cc] -= f * M[c * m + cc];
      r[rr] -= f * r[c];
    }
  }
  x.assign(m, 0.0);
  for (int c = m - 1; c >= 0; --c) {
    double acc = r[c];
    for (int cc = c + 1; cc < m; ++cc) acc -= M[c * m + cc] * x[cc];
    x[c] = acc / M[c * m + c];
  }
  return true;
}

// Solves (Delta + L) x = g, L(i,j) = scale_i * A(i,j) for j in J_i, block by
// block in plan order: a single cell is a scalar update, a coupled block is a
// small dense system (the paper's local systems).
// transpose=true solves (Delta + L^T) x = g instead (the backward half of the
// symmetric SSOR apply): blocks in reverse order, L^T(i,j) = L(j,i).
bool block_solve(const Problem& pb, const Plan& pl, const double* Delta, const double* scale,
                 const double* gvec, double* x, bool transpose, const double* E = nullptr) {
  // E: the entries to use instead of A's (s x N, diagonal-major), or null
  auto ent = [&](int k, int64_t i) { return E ? E[(size_t)k * pb.g.N + i] : aval(pb, k, i); };
  const Grid& g = pb.g;
  const int64_t nb = (int64_t)pl.bstart.size() - 1;
  std::vector<double> M, r, sol;
  for (int64_t bb = 0; bb < nb; ++bb) {
    const int64_t b = transpose ? (nb - 1 - bb) : bb;
    const int64_t b0 = pl.bstart[b], b1 = pl.bstart[b + 1];
    const int m = (int)(b1 - b0);
    auto pos = [&](int64_t j) -> int {
      for (int p = 0; p < m; ++p)
        if (pl.order[b0 + p] == j) return p;
      return -1;
    };
    M.assign((size_t)m * m, 0.0);
    r.assign(m, 0.0);
    for (int p = 0; p < m; ++p) {
      const int64_t i = pl.order[b0 + p];
      M[p * m + p] = Delta[i];
      double acc = gvec[i];
      for (int k = 1; k < g.s; ++k) {
        const int64_t j = neighbour(g, i, k);
        if (j < 0) continue;
        double coef;
        if (!transpose) {
          if (!(pl.jmask[i] >> k & 1)) continue;
          coef = (scale ? scale[i] : 1.0) * ent(k, i);
        } else {
          const int kb = g.opp[k];  // entry of row j that points back to i
          if (!(pl.jmask[j] >> kb & 1)) continue;
          coef = (scale ? scale[j] : 1.0) * ent(kb, j);
        }
        const int c = pos(j);
        if (c >= 0) M[p * m + c] += coef;
        else acc -= coef * x[j];
      }
      r[p] = acc;
    }
    if (m == 1) {
      x[pl.order[b0]] = r[0] / M[0];
    } else {
      if (!dense_solve(m, M, r, sol)) return false;
      for (int p = 0; p < m; ++p) x[pl.order[b0 + p]] = sol[p];
    }
  }
  return true;
}

// y = A x (Eq. d2d applied as a matrix).
void matvec(const Problem& pb, const double* x, double* y) {
  const Grid& g = pb.g;
  for (int64_t i = 0; i < g.N; ++i) {
    double acc = aval(pb, 0, i) * x[i];
    for (int k = 1; k < g.s; ++k) {
      const int64_t j = neighbour(g, i, k);
      if (j >= 0) acc += aval(pb, k, i) * x[j];
    }
    y[i] = acc;
  }
}

double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

// One SOR sweep of the decomposed (or natural) ordering, in the splitting form
// of Eq. (ca2d:matiter):  (D + w L_J) u+ = ((1-w) D - w U_J) u + w b,
// with w = omega[start corner of the row's subdomain] (one relaxation factor
// per sweep direction, Sec. 3: w_SW, w_NE, w_SE, w_NW; Sec. 4: eight in 3D).
bool sor_sweep(Problem& pb, int mode, int64_t t, const double* omega, const double* b,
               const double* u, double* unew) {
  const Grid& g = pb.g;
  Plan& pl = get_plan(pb, mode, t);
  std::vector<double> w(g.N), Dg(g.N), rhs(g.N);
  for (int64_t i = 0; i < g.N; ++i) {
    const double wi = omega[pl.corner[i]];
    w[i] = wi;
    const double aii = aval(pb, 0, i);
    Dg[i] = aii;
    double acc = (1.0 - wi) * aii * u[i] + wi * b[i];
    for (int k = 1; k < g.s; ++k) {
      if (pl.jmask[i] >> k & 1) continue;
      const int64_t j = neighbour(g, i, k);
      if (j >= 0) acc -= wi * aval(pb, k, i) * u[j];
    }
    rhs[i] = acc;
  }
  return block_solve(pb, pl, Dg.data(), w.data(), rhs.data(), unew, false);
}

// Forward phase of the preconditioners: the phase at which subdomain (0,0,0)
// sweeps from its origin corner, so that with one subdomain the forward solve
// is the natural (lexicographic) one. Its reverse phase is t ^ 1.
int64_t fwd_phase(int d) { return d == 1 ? 0 : 1; }

// ILU(0), Sec. 5: one symmetric Gauss-Seidel pass on an n-diagonal matrix is
// ILU(0) (Saad, Sec. 10.3).
//  natural:    Saad's IKJ ILU(0) restricted to the pattern of A.
//  decomposed: M = (D~ + L_J) D~^-1 (D~ + U_J), L_J = implicit entries of the
//              forward phase, U_J = implicit entries of its reverse phase, and
//              d~_i = a_ii - sum_{j in J_i, i not in J_j} a_ij a_ji / d~_j.
bool ilu0_factor_full(Problem& pb);

bool ilu0_factor(Problem& pb, int mode) {
  const Grid& g = pb.g;
  const int64_t N = g.N;
  pb.ilu_mode = mode;
  if (mode == MODE_DECOMPOSED_FULL) return ilu0_factor_full(pb);
  if (mode == MODE_DECOMPOSED) {
    Plan& pl = get_plan(pb, MODE_DECOMPOSED, fwd_phase(g.d));
    pb.dtilde.assign(N, 0.0);
    const int64_t nb = (int64_t)pl.bstart.size() - 1;
    for (int64_t b = 0; b < nb; ++b) {
      for (int64_t p = pl.bstart[b]; p < pl.bstart[b + 1]; ++p) {
        const int64_t i = pl.order[p];
        double acc = aval(pb, 0, i);
        for (int k = 1; k < g.s; ++k) {
          if (!(pl.jmask[i] >> k & 1)) continue;
          const int64_t j = neighbour(g, i, k);
          const int kb = g.opp[k];
          if (pl.jmask[j] >> kb & 1) continue;  // mutual pair: no elimination term
          // j precedes i in a strictly earlier block (checked below).
          bool in_block = false;
          for (int64_t q = pl.bstart[b]; q < pl.bstart[b + 1]; ++q)
            if (pl.order[q] == j) in_block = true;
          if (in_block) return false;
          acc -= aval(pb, k, i) * aval(pb, kb, j) / pb.dtilde[j];
        }
        if (acc == 0.0) return false;
        pb.dtilde[i] = acc;
      }
    }
    get_plan(pb, MODE_DECOMPOSED, fwd_phase(g.d) ^ 1);
    return true;
  }
  // Natural IKJ ILU(0) on the pattern (Saad Alg. 10.4). Row i holds entries
  // k = 0..s-1 (A(i, i+off_k)); columns are compared by natural index.
  pb.lu = pb.A;
  auto L = [&](int k, int64_t i) -> double& { return pb.lu[(size_t)k * N + i]; };
  for (int64_t i = 0; i < N; ++i) {
    // entries of row i sorted by column
    int ks[9];
    int64_t cols[9];
    int m = 0;
    for (int k = 0; k < g.s; ++k) {
      const int64_t j = (k == 0) ? i : neighbour(g, i, k);
      if (j < 0) continue;
      ks[m] = k;
      cols[m] = j;
      ++m;
    }
    for (int a = 0; a < m; ++a)
      for (int b2 = a + 1; b2 < m; ++b2)
        if (cols[b2] < cols[a]) {
          std::swap(cols[a], cols[b2]);
          std::swap(ks[a], ks[b2]);
        }
    for (int a = 0; a < m; ++a) {
      const int64_t kc = cols[a];
      if (kc >= i) break;
      // a_ik := a_ik / a_kk
      L(ks[a], i) /= L(0, kc);
      const double lik = L(ks[a], i);
      // for j > k in row i's pattern: a_ij -= a_ik * a_kj (if (k,j) in pattern)
      for (int b2 = a + 1; b2 < m; ++b2) {
        const int64_t j = cols[b2];
        // find entry of row kc pointing to j
        for (int kk = 0; kk < g.s; ++kk) {
          const int64_t jj = (kk == 0) ? kc : neighbour(g, kc, kk);
          if (jj == j) {
            L(ks[b2], i) -= lik * L(kk, kc);
            break;
          }
        }
      }
    }
    if (L(0, i) == 0.0) return false;
  }
  return true;
}

// Decomposed full ILU(0) on the stencil's pattern (the 9-point molecule keeps
// the elimination's updates of off-diagonal entries; Sec. 5 read as the ILU(0)
// of every subdomain's diagonal block in the order its sweep visits it):
// within every subdomain, the IKJ elimination (Saad Alg. 10.4) of A's
// diagonal block in that subdomain's own order at the forward phase (its
// reflected lexicographic order, the order of its sweep); entries that point
// into another subdomain stay A's, and the apply couples across interfaces
// exactly as the decomposed sweep does (mutual face pairs, Sec. 3). The factor
// is kept as F (s x N) in the form M = (D + L') D^-1 (D + U'): F(0, i) = u_ii,
// lower entries l_ij u_jj, upper entries u_ij. With one subdomain this is the
// natural IKJ ILU(0); on 5/7-point matrices nothing but the pivots changes.
bool ilu0_factor_full(Problem& pb) {
  const Grid& g = pb.g;
  const int64_t N = g.N;
  const Plan& pl = get_plan(pb, MODE_DECOMPOSED, fwd_phase(g.d));
  pb.full = pb.A;
  auto F = [&](int k, int64_t i) -> double& { return pb.full[(size_t)k * N + i]; };
  // the cells of every subdomain, each in its own sweep order
  std::vector<int64_t> cells(N);
  for (int64_t i = 0; i < N; ++i) cells[i] = i;
  auto sub_of = [&](int64_t i) {
    int64_t c[3];
    coords(g, i, c);
    return pb.P.part_of[0][c[0]] + (int64_t)pb.P.p[0] *
           (pb.P.part_of[1][c[1]] + (int64_t)pb.P.p[1] * pb.P.part_of[2][c[2]]);
  };
  std::stable_sort(cells.begin(), cells.end(), [&](int64_t a, int64_t b) {
    const int64_t sa = sub_of(a), sb = sub_of(b);
    if (sa != sb) return sa < sb;
    int64_t ca[3], cb[3];
    coords(g, a, ca);
    coords(g, b, cb);
    return precedes(ca, cb, pl.corner[a]);
  });
  for (int64_t i : cells) {
    int64_t ci[3];
    coords(g, i, ci);
    const int cs = pl.corner[i];
    // entries of row i inside its subdomain, in the subdomain's order
    int ks[27];
    int64_t cols[27];
    int m = 0;
    for (int k = 0; k < g.s; ++k) {
      const int64_t j = (k == 0) ? i : neighbour(g, i, k);
      if (j < 0) continue;
      int64_t cj[3];
      coords(g, j, cj);
      if (!same_part(pb, ci, cj)) continue;
      ks[m] = k;
      cols[m] = j;
      ++m;
    }
    auto before = [&](int64_t a, int64_t b) {
      int64_t ca[3], cb[3];
      coords(g, a, ca);
      coords(g, b, cb);
      return precedes(ca, cb, cs);
    };
    for (int a = 0; a < m; ++a)
      for (int b2 = a + 1; b2 < m; ++b2)
        if (before(cols[b2], cols[a])) {
          std::swap(cols[a], cols[b2]);
          std::swap(ks[a], ks[b2]);
        }
    int nlow = 0;
    for (int a = 0; a < m && cols[a] != i; ++a) {
      const int64_t kc = cols[a];
      ++nlow;
      // a_ik := a_ik / a_kk
      F(ks[a], i) /= F(0, kc);
      const double lik = F(ks[a], i);
      // every later entry j of row i that row k holds: a_ij -= a_ik a_kj
      for (int b2 = a + 1; b2 < m; ++b2) {
        const int64_t j = cols[b2];
        for (int kk = 0; kk < g.s; ++kk) {
          const int64_t jj = (kk == 0) ? kc : neighbour(g, kc, kk);
          if (jj == j) {
            F(ks[b2], i) -= lik * F(kk, kc);
            break;
          }
        }
      }
    }
    if (F(0, i) == 0.0) return false;
    for (int a = 0; a < nlow; ++a) F(ks[a], i) *= F(0, cols[a]);  // l_ij u_jj
  }
  get_plan(pb, MODE_DECOMPOSED, fwd_phase(g.d) ^ 1);
  return true;
}

bool ilu0_apply(Problem& pb, const double* r, double* z) {
  const Grid& g = pb.g;
  const int64_t N = g.N;
  if (pb.ilu_mode == MODE_DECOMPOSED_FULL) {
    const int64_t tf = fwd_phase(g.d);
    Plan& pf = get_plan(pb, MODE_DECOMPOSED, tf);
    Plan& pbk = get_plan(pb, MODE_DECOMPOSED, tf ^ 1);
    const double* E = pb.full.data();
    std::vector<double> d(E, E + N), y(N), dy(N);
    // (D + L') y = r ; (D + U') z = D y, each with the decomposed sweep's couplings
    if (!block_solve(pb, pf, d.data(), nullptr, r, y.data(), false, E)) return false;
    for (int64_t i = 0; i < N; ++i) dy[i] = d[i] * y[i];
    return block_solve(pb, pbk, d.data(), nullptr, dy.data(), z, false, E);
  }
  if (pb.ilu_mode == MODE_DECOMPOSED) {
    const int64_t tf = fwd_phase(g.d);
    Plan& pf = get_plan(pb, MODE_DECOMPOSED, tf);
    Plan& pbk = get_plan(pb, MODE_DECOMPOSED, tf ^ 1);
    std::vector<double> y(N), dy(N);
    // (D~ + L_J) y = r
    if (!block_solve(pb, pf, pb.dtilde.data(), nullptr, r, y.data(), false)) return false;
    // (D~ + U_J) z = D~ y, U_J = implicit entries of the reverse phase
    for (int64_t i = 0; i < N; ++i) dy[i] = pb.dtilde[i] * y[i];
    return block_solve(pb, pbk, pb.dtilde.data(), nullptr, dy.data(), z, false);
  }
  if (pb.ilu_mode == MODE_NATURAL) {
    auto L = [&](int k, int64_t i) -> double { return pb.lu[(size_t)k * N + i]; };
    std::vector<double> y(N);
    for (int64_t i = 0; i < N; ++i) {
      double acc = r[i];
      for (int k = 1; k < g.s; ++k) {
        const int64_t j = neighbour(g, i, k);
        if (j >= 0 && j < i) acc -= L(k, i) * y[j];
      }
      y[i] = acc;
    }
    for (int64_t i = N - 1; i >= 0; --i) {
      double acc = y[i];
      for (int k = 1; k < g.s; ++k) {
        const int64_t j = neighbour(g, i, k);
        if (j > i) acc -= L(k, i) * z[j];
      }
      z[i] = acc / L(0, i);
    }
    return true;
  }
  return false;
}

// Symmetric SSOR apply (SPD form, usable inside CG):
//   z = w(2-w) (D + w L_J^T)^-1 D (D + w L_J)^-1 r,
// L_J = implicit entries of the forward phase. With one subdomain this is the
// classical SSOR preconditioner (forward sweep then backward sweep, Sec. 2).
bool ssor_apply(Problem& pb, int mode, double omega, const double* r, double* z) {
  const Grid& g = pb.g;
  const int64_t N = g.N;
  Plan& pl = get_plan(pb, mode, fwd_phase(g.d));
  std::vector<double> Dg(N), w(N, omega), v(N), t(N);
  for (int64_t i = 0; i < N; ++i) Dg[i] = aval(pb, 0, i);
  if (!block_solve(pb, pl, Dg.data(), w.data(), r, t.data(), false)) return false;
  for (int64_t i = 0; i < N; ++i) v[i] = Dg[i] * t[i];
  if (!block_solve(pb, pl, Dg.data(), w.data(), v.data(), z, true)) return false;
  const double f = omega * (2.0 - omega);
  for (int64_t i = 0; i < N; ++i) z[i] *= f;
  return true;
}

enum { PREC_NONE = 0, PREC_SSOR = 1, PREC_ILU0 = 2 };
enum { METHOD_PCG = 0, METHOD_BICGSTAB = 1, METHOD_STATIONARY = 2 };

bool precond(Problem& pb, int prec, int mode, double omega, const double* r, double* z) {
  const int64_t N = pb.g.N;
  if (prec == PREC_NONE) {
    std::memcpy(z, r, sizeof(double) * N);
    return true;
  }
  if (prec == PREC_SSOR) return ssor_apply(pb, mode, omega, r, z);
  if (prec == PREC_ILU0) return ilu0_apply(pb, r, z);
  return false;
}

double true_relres(Problem& pb, const double* b, const double* x, double bnorm, std::vector<double>& tmp) {
  const int64_t N = pb.g.N;
  tmp.resize(N);
  matvec(pb, x, tmp.data());
  for (int64_t i = 0; i < N; ++i) tmp[i] = b[i] - tmp[i];
  return std::sqrt(dot(N, tmp.data(), tmp.data())) / bnorm;
}

// Krylov drivers. x starts from the given x. Stop rule shared with the GPU
// library: the recurrence residual ||r||/||b|| <= rtol triggers a check of the
// true residual b - A x; if that is above rtol the method restarts from it.
// info[0] = iterations, info[1] = final true relative residual, info[2] = status
// (0 converged, 1 not converged, 2 breakdown).
int pcg(Problem& pb, int prec, int mode, double omega, double rtol, int maxit, const double* b,
        double* x, double* info) {
  const int64_t N = pb.g.N;
  std::vector<double> r(N), z(N), p(N), Ap(N), tmp;
  const double bnorm = std::sqrt(dot(N, b, b));
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
    info[0] = 0; info[1] = 0; info[2] = 0;
    return 0;
  }
  int it = 0;
  for (;;) {  // (re)start from the true residual
    matvec(pb, x, Ap.data());
    for (int64_t i = 0; i < N; ++i) r[i] = b[i] - Ap[i];
    double rel = std::sqrt(dot(N, r.data(), r.data())) / bnorm;
    if (rel <= rtol) { info[0] = it; info[1] = rel; info[2] = 0; return 0; }
    if (!precond(pb, prec, mode, omega, r.data(), z.data())) return 3;
    p = z;
    double rz = dot(N, r.data(), z.data());
    bool recheck = false;
    while (it < maxit) {
      matvec(pb, p.data(), Ap.data());
      const double pAp = dot(N, p.data(), Ap.data());
      if (pAp == 0.0 || rz == 0.0) { info[0] = it; info[1] = true_relres(pb, b, x, bnorm, tmp); info[2] = 2; return 0; }
      const double alpha = rz / pAp;
      for (int64_t i = 0; i < N; ++i) x[i] += alpha * p[i];
      for (int64_t i = 0; i < N; ++i) r[i] -= alpha * Ap[i];
      ++it;
      const double rrel = std::sqrt(dot(N, r.data(), r.data())) / bnorm;
      pb.hist.insert(pb.hist.end(), {rrel, alpha, 0.0, 0.0});
      if (rrel <= rtol) { recheck = true; break; }
      if (!precond(pb, prec, mode, omega, r.data(), z.data())) return 3;
      const double rz2 = dot(N, r.data(), z.data());
      const double beta = rz2 / rz;
      rz = rz2;
      for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (!recheck) { info[0] = it; info[1] = true_relres(pb, b, x, bnorm, tmp); info[2] = 1; return 0; }
    const double tr = true_relres(pb, b, x, bnorm, tmp);
    if (tr <= rtol) { info[0] = it; info[1] = tr; info[2] = 0; return 0; }
  }
}

// Right-preconditioned BiCGSTAB (van der Vorst 1992), same stop rule as pcg.
int bicgstab(Problem& pb, int prec, int mode, double omega, double rtol, int maxit,
             const double* b, double* x, double* info) {
  const int64_t N = pb.g.N;
  std::vector<double> r(N), rh(N), p(N), v(N), ph(N), s(N), sh(N), t(N), tmp;
  const double bnorm = std::sqrt(dot(N, b, b));
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
    info[0] = 0; info[1] = 0; info[2] = 0;
    return 0;
  }
  int it = 0;
  for (;;) {
    matvec(pb, x, t.data());
    for (int64_t i = 0; i < N; ++i) r[i] = b[i] - t[i];
    double rel = std::sqrt(dot(N, r.data(), r.data())) / bnorm;
    if (rel <= rtol) { info[0] = it; info[1] = rel; info[2] = 0; return 0; }
    rh = r;
    double rho_old = 1.0, alpha = 1.0, om = 1.0;
    std::fill(v.begin(), v.end(), 0.0);
    std::fill(p.begin(), p.end(), 0.0);
    bool recheck = false;
    while (it < maxit) {
      const double rho = dot(N, rh.data(), r.data());
      if (rho == 0.0 || om == 0.0) { info[0] = it; info[1] = true_relres(pb, b, x, bnorm, tmp); info[2] = 2; return 0; }
      const double beta = (rho / rho_old) * (alpha / om);
      rho_old = rho;
      for (int64_t i = 0; i < N; ++i) p[i] = r[i] + beta * (p[i] - om * v[i]);
      if (!precond(pb, prec, mode, omega, p.data(), ph.data())) return 3;
      matvec(pb, ph.data(), v.data());
      const double rv = dot(N, rh.data(), v.data());
      if (rv == 0.0) { info[0] = it; info[1] = true_relres(pb, b, x, bnorm, tmp); info[2] = 2; return 0; }
      alpha = rho / rv;
      for (int64_t i = 0; i < N; ++i) s[i] = r[i] - alpha * v[i];
      ++it;
      const double srel = std::sqrt(dot(N, s.data(), s.data())) / bnorm;
      if (srel <= rtol) {  // the half step meets the tolerance: x += alpha ph, r = s
        for (int64_t i = 0; i < N; ++i) x[i] += alpha * ph[i];
        pb.hist.insert(pb.hist.end(), {srel, srel, alpha, 0.0});
        recheck = true;
        break;
      }
      if (!precond(pb, prec, mode, omega, s.data(), sh.data())) return 3;
      matvec(pb, sh.data(), t.data());
      const double tt = dot(N, t.data(), t.data());
      om = (tt == 0.0) ? 0.0 : dot(N, t.data(), s.data()) / tt;
      for (int64_t i = 0; i < N; ++i) x[i] += alpha * ph[i] + om * sh[i];
      for (int64_t i = 0; i < N; ++i) r[i] = s[i] - om * t[i];
      const double rrel = std::sqrt(dot(N, r.data(), r.data())) / bnorm;
      pb.hist.insert(pb.hist.end(), {srel, rrel, alpha, om});
      if (rrel <= rtol) { recheck = true; break; }
    }
    if (!recheck) { info[0] = it; info[1] = true_relres(pb, b, x, bnorm, tmp); info[2] = 1; return 0; }
    const double tr = true_relres(pb, b, x, bnorm, tmp);
    if (tr <= rtol) { info[0] = it; info[1] = tr; info[2] = 0; return 0; }
  }
}

// Stationary iteration: sweep t = 0, 1, 2, ... of the schedule (Sec. 2-4),
// stopping at the first iterate with ||b - A x||/||b|| <= rtol.
int stationary(Problem& pb, int mode, const double* omega, double rtol, int maxit,
               const double* b, double* x, double* info) {
  const int64_t N = pb.g.N;
  std::vector<double> xn(N), tmp;
  double bnorm = std::sqrt(dot(N, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
  double rel = true_relres(pb, b, x, bnorm, tmp);
  int it = 0;
  while (rel > rtol && it < maxit) {
    if (!sor_sweep(pb, mode, it, omega, b, x, xn.data())) return 3;
    std::memcpy(x, xn.data(), sizeof(double) * N);
    ++it;
    rel = true_relres(pb, b, x, bnorm, tmp);
  }
  info[0] = it;
  info[1] = rel;
  info[2] = (rel <= rtol) ? 0 : 1;
  return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// Fast sweeping for the eikonal equation |grad u| = f on a 2D grid of spacing
// h. The paper's closing remarks name the fast sweeping method as another
// sequential sweep that its decomposition parallelises (details only in its
// supplement, which is not available); the local update is the Godunov upwind
// discretisation of Zhao's fast sweeping method (H.-K. Zhao, Math. Comp. 74,
// 2005):
//   a = min(u_W, u_E), b = min(u_S, u_N)        (outside the grid: +inf)
//   |a - b| >= f h :  u~ = min(a, b) + f h
//   otherwise      :  u~ = (a + b + sqrt(2 (f h)^2 - (a - b)^2)) / 2
//   u <- min(u, u~)
// Sources are cells with u = 0 initially (the min keeps them), all others
// start at +inf.
// One decomposed sweep at phase t: every subdomain runs a Gauss-Seidel pass
// from its start corner, the schedule of the linear sweeps (subdomain_corner);
// inside the subdomain, cells already visited give their new values and the
// rest their old ones; cells of other subdomains always give old values (the
// halo of old values, Sec. 3 "Data structure"). With one subdomain the four
// consecutive phases are Zhao's four alternating orderings.
// Stop rule: sweeps run in rounds of four phases; the solve ends after the
// first round whose largest change |u_new - u_old| over its sweeps is <= delta.
// ---------------------------------------------------------------------------
double eik_update(double a, double b, double fh) {
  const double d = a - b;
  if (!(std::fabs(d) < fh)) return std::min(a, b) + fh;
  return (a + b + std::sqrt(2.0 * (fh * fh) - d * d)) * 0.5;
}

struct Eik {
  Grid g;
  Partition P;
  double h = 0.0;
  std::vector<double> f;
};

// One decomposed sweep; returns the largest |u_new - u_old|.
double eik_sweep(const Eik& E, int64_t t, const double* uo, double* un) {
  const Grid& g = E.g;
  const int64_t nx = g.n[0], ny = g.n[1];
  const double inf = std::numeric_limits<double>::infinity();
  std::copy(uo, uo + g.N, un);
  for (int iy = 0; iy < E.P.p[1]; ++iy)
    for (int ix = 0; ix < E.P.p[0]; ++ix) {
      const int idx[3] = {ix, iy, 0};
      const int c = subdomain_corner(2, t, idx);
      const int64_t x0 = E.P.lo[0][ix], x1 = E.P.lo[0][ix + 1];
      const int64_t y0 = E.P.lo[1][iy], y1 = E.P.lo[1][iy + 1];
      // value of cell (x, y) as seen from this subdomain's pass
      auto val = [&](int64_t x, int64_t y) -> double {
        if (x < 0 || x >= nx || y < 0 || y >= ny) return inf;
        const bool mine = x >= x0 && x < x1 && y >= y0 && y < y1;
        return mine ? un[y * nx + x] : uo[y * nx + x];
      };
      for (int64_t yy = 0; yy < y1 - y0; ++yy) {
        const int64_t y = (c & 2) ? y1 - 1 - yy : y0 + yy;
        for (int64_t xx = 0; xx < x1 - x0; ++xx) {
          const int64_t x = (c & 1) ? x1 - 1 - xx : x0 + xx;
          const int64_t i = y * nx + x;
          const double a = std::min(val(x - 1, y), val(x + 1, y));
          const double b = std::min(val(x, y - 1), val(x, y + 1));
          un[i] = std::min(un[i], eik_update(a, b, E.f[i] * E.h));
        }
      }
    }
  double m = 0.0;
  for (int64_t i = 0; i < g.N; ++i)
    if (un[i] != uo[i]) m = std::max(m, uo[i] - un[i]);  // values only decrease
  return m;
}

// ---------------------------------------------------------------------------
// C interface (loaded with ctypes by the tests). Return 0 on success.
// ---------------------------------------------------------------------------
extern "C" {

void* orc_create(int d, const int64_t* n, int stencil, const double* diags, const int* sub) {
  Problem* pb = new Problem();
  if (!make_grid(pb->g, d, n, stencil) || !make_partition(pb->g, sub, pb->P)) {
    delete pb;
    return nullptr;
  }
  pb->A.assign(diags, diags + (size_t)stencil * pb->g.N);
  return pb;
}

void orc_destroy(void* h) { delete static_cast<Problem*>(h); }

int64_t orc_ncells(void* h) { return static_cast<Problem*>(h)->g.N; }

int orc_base_corner(int d, int64_t t) { return base_corner(d, t); }

int orc_matvec(void* h, const double* x, double* y) {
  matvec(*static_cast<Problem*>(h), x, y);
  return 0;
}

// Exports J_i (bit k of out[i]) and the start corner of every cell's
// subdomain at phase t; returns the number of coupled blocks and the largest.
int orc_plan_info(void* h, int mode, int64_t t, uint16_t* jmask, uint8_t* corner,
                  int64_t* nblocks, int64_t* maxblock) {
  Problem& pb = *static_cast<Problem*>(h);
  Plan& pl = get_plan(pb, mode, t);
  if (jmask) std::memcpy(jmask, pl.jmask.data(), sizeof(uint16_t) * pb.g.N);
  if (corner) std::memcpy(corner, pl.corner.data(), pb.g.N);
  const int64_t nb = (int64_t)pl.bstart.size() - 1;
  int64_t mx = 0;
  for (int64_t b = 0; b < nb; ++b) mx = std::max<int64_t>(mx, pl.bstart[b + 1] - pl.bstart[b]);
  if (nblocks) *nblocks = nb;
  if (maxblock) *maxblock = mx;
  return 0;
}

int orc_sor_sweep(void* h, int mode, int64_t t, const double* omega, const double* b,
                  const double* x_old, double* x_new) {
  return sor_sweep(*static_cast<Problem*>(h), mode, t, omega, b, x_old, x_new) ? 0 : 1;
}

int orc_ilu0_factor(void* h, int mode) {
  return ilu0_factor(*static_cast<Problem*>(h), mode) ? 0 : 1;
}

// Decomposed: out[0..N) = d~. Natural: out[0..s*N) = L multipliers (entries
// pointing to lower indices) and U (diagonal and upper entries), diagonal-major.
// Decomposed full: out[0..s*N) = F, diagonal u_ii, lower entries l_ij u_jj,
// upper entries u_ij (lower/upper in the subdomain's sweep order; entries
// into another subdomain are A's).
int orc_ilu0_export(void* h, double* out) {
  Problem& pb = *static_cast<Problem*>(h);
  if (pb.ilu_mode == MODE_DECOMPOSED) {
    std::memcpy(out, pb.dtilde.data(), sizeof(double) * pb.g.N);
    return 0;
  }
  if (pb.ilu_mode == MODE_NATURAL) {
    std::memcpy(out, pb.lu.data(), sizeof(double) * pb.lu.size());
    return 0;
  }
  if (pb.ilu_mode == MODE_DECOMPOSED_FULL) {
    std::memcpy(out, pb.full.data(), sizeof(double) * pb.full.size());
    return 0;
  }
  return 1;
}

int orc_ilu0_apply(void* h, const double* r, double* z) {
  return ilu0_apply(*static_cast<Problem*>(h), r, z) ? 0 : 1;
}

int orc_ssor_apply(void* h, int mode, double omega, const double* r, double* z) {
  return ssor_apply(*static_cast<Problem*>(h), mode, omega, r, z) ? 0 : 1;
}

int orc_fwd_phase(int d) { return (int)fwd_phase(d); }

void* orc_eik_create(const int64_t* n, double h, const double* f, const int* sub) {
  Eik* E = new Eik();
  const int64_t n3[3] = {n[0], n[1], 1};
  const int sub3[3] = {sub[0], sub[1], 1};
  if (!(h > 0.0) || !make_grid(E->g, 2, n3, 5) || !make_partition(E->g, sub3, E->P)) {
    delete E;
    return nullptr;
  }
  E->h = h;
  E->f.assign(f, f + E->g.N);
  return E;
}

void orc_eik_destroy(void* e) { delete static_cast<Eik*>(e); }

// one sweep at phase t; *change = largest |u_new - u_old|
int orc_eik_sweep(void* e, int64_t t, const double* uo, double* un, double* change) {
  *change = eik_sweep(*static_cast<Eik*>(e), t, uo, un);
  return 0;
}

// rounds of four sweeps (phases 0, 1, 2, 3, 4, ...) from u until a round's
// largest change is <= delta; u receives the result; info = {sweeps, last
// round's largest change, converged}
int orc_eik_solve(void* e, double* u, double delta, int max_rounds, double* info) {
  Eik& E = *static_cast<Eik*>(e);
  std::vector<double> a(u, u + E.g.N), b(E.g.N);
  int64_t t = 0;
  double m = 0.0;
  bool done = false;
  for (int r = 0; r < max_rounds && !done; ++r) {
    m = 0.0;
    for (int k = 0; k < 4; ++k, ++t) {
      m = std::max(m, eik_sweep(E, t, a.data(), b.data()));
      a.swap(b);
    }
    done = m <= delta;
  }
  std::copy(a.begin(), a.end(), u);
  info[0] = (double)t;
  info[1] = m;
  info[2] = done ? 1.0 : 0.0;
  return 0;
}

int orc_solve(void* h, int method, int prec, int mode, const double* omega, double rtol,
              int maxit, const double* b, double* x, double* info) {
  Problem& pb = *static_cast<Problem*>(h);
  pb.hist.clear();
  // an ILU(0) solve keeps the factor it finds in the same ordering (the full
  // decomposed factor too); otherwise it factors first
  const bool have = pb.ilu_mode == mode || (mode == MODE_DECOMPOSED && pb.ilu_mode == MODE_DECOMPOSED_FULL);
  if (prec == PREC_ILU0 && !have)
    if (!ilu0_factor(pb, mode)) return 4;
  switch (method) {
    case METHOD_PCG: return pcg(pb, prec, mode, omega[0], rtol, maxit, b, x, info);
    case METHOD_BICGSTAB: return bicgstab(pb, prec, mode, omega[0], rtol, maxit, b, x, info);
    case METHOD_STATIONARY: return stationary(pb, mode, omega, rtol, maxit, b, x, info);
  }
  return 5;
}

// Rows (4 values each) of the last solve's per-iteration record copied to out,
// at most cap; returns the number of rows the solve recorded.
int64_t orc_history(void* h, double* out, int64_t cap) {
  const Problem& pb = *static_cast<Problem*>(h);
  const int64_t rows = (int64_t)pb.hist.size() / 4;
  const int64_t n = std::min(rows, cap);
  if (out && n > 0) std::memcpy(out, pb.hist.data(), sizeof(double) * 4 * (size_t)n);
  return rows;
}

}  // extern "C"
