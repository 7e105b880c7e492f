// FP64 CPU oracle for the APIC augury contact step (Tupek, Koester, Mosby,
// "A momentum preserving frictional contact algorithm based on affine
// particle-in-cell grid transfers", arXiv 2108.02259).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// definition that the CUDA library is checked against.  Only the test suite,
// the smoke check and the CPU-baseline leg of the benchmark may load it.  It
// shares no code, header or constant with the CUDA library.
//
// Everything is double precision, the background grid is an unbounded
// hash map keyed by integer node coordinates, and every step follows the
// paper's equations in the paper's order:
//   * quadratic B-spline weights ............ App. B (with the 1/4 reading of
//                                              the two middle functions)
//   * D_p = sum_i N_i (x_i - x_p) (x) (x_i - x_p)   Sec. 2.1.2 (computed, not assumed)
//   * mass / APIC momentum P2G .............. Sec. 2.1.1 eq. massToGrid,
//                                              Sec. 2.1.2 eq. particleToGrid
//   * APIC G2P, B_p .......................... eq. gridToParticle, eq. scaledVelGrad
//   * augury series V + G V + sum G W_n ...... Sec. 2.3
//   * undesirable part (Coulomb friction) ..... Sec. 2.4 (default) or the
//                                              Sec. 2.3 separation rule (flag)
//   * 1-D two-particle linear-hat transfers ... Sec. 3.1
//   * node normals from boundary faces ....... Sec. 2.3 (area-weighted)
//   * normals from a body's grid mass ........ a reading for callers with no
//                                              surface mesh (App. B weights
//                                              and their derivatives)
//   * augury dynamics, springs + gravity ...... Sec. 2.2 eq. apic_accel,
//                                              eq. Newmark (velocity Verlet)
//
// The public C ABI takes C_p = B_p D_p^{-1} (the APIC affine matrix) because
// that is what callers carry; internally B_p = C_p D_p with D_p computed from
// the weights, so the oracle never hard-codes D_p = (h^2/2) I.
//
// Parity status per function (see the tests for the pins):
//   oracle_weights ................ pinned (partition of unity, linear
//                                    completeness, D = h^2/2 I, printed values)
//   oracle_apply_H / p2g_grid ..... pinned (affine reproduction, momentum,
//                                    dense brute force, quasi-null space)
//   oracle_undesirable ............ pinned (closed-form cone cases)
//   oracle_contact_step ........... pinned (momentum, affine, symmetry)
//   oracle_apic1d_linear .......... pinned (closed-form matrix of Sec. 3.1)
//   oracle_node_normals ........... pinned (closed-form cube, roof and
//                                    plane cases, icosahedron symmetry,
//                                    winding and rotation)
//   oracle_augury_steps ........... pinned (discrete Verlet closed forms for
//                                    an isolated spring pair and free fall,
//                                    rigid translation, momentum, mirror
//                                    symmetry); rebound threshold unpinned
//   oracle_mass_normals ........... pinned (weight-derivative identities and
//                                    finite differences, exact face normals
//                                    of grid-aligned lattice boxes, zero in
//                                    the interior, integer-shift and axis
//                                    invariance, bodies independent); the
//                                    threshold itself is a reading
//   per-body-pair friction (mu_pair) ... parity unpinned (a reading; the paper
//                                    has a single scalar mu)
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

// Flags; the values are part of the oracle's own ABI.
constexpr uint32_t ORC_PIC = 1u << 0;    // PIC transfers: no affine term (D_p = 0)
constexpr uint32_t ORC_SEP23 = 1u << 1;  // Sec. 2.3 separation rule instead of Sec. 2.4

struct Key {
  int64_t i, j, k;
  bool operator==(const Key& o) const { return i == o.i && j == o.j && k == o.k; }
};
struct KeyHash {
  size_t operator()(const Key& a) const {
    uint64_t h = (uint64_t)a.i * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)a.j * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)a.k * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

// App. B: the grid point to the left of xi = x/h is i = floor(xi); the four
// functions covering xi are N_{i-1}, N_i, N_{i+1}, N_{i+2}, built from
// a_i, b_i, c_i.  The printed factor 1/8 on the middle two violates the
// partition of unity the appendix itself requires (eq. pou); 1/4 restores it
// together with linear completeness and D_p = (h^2/2) I.
void weights_1d(double xi, int64_t* ileft, double N[4]) {
  const double fi = std::floor(xi);
  const int64_t i = (int64_t)fi;
  const double a = (fi + 1.0 - xi) * (fi + 1.0 - xi);
  const double b = (-fi + 1.0 + xi) * (fi + 1.0 - xi) + (fi + 2.0 - xi) * (xi - fi);
  const double c = (xi - fi) * (xi - fi);
  N[0] = 0.25 * a;
  N[1] = 0.25 * (a + b);
  N[2] = 0.25 * (b + c);
  N[3] = 0.25 * c;
  *ileft = i;
}

// Derivatives dN_k/dxi of the four App. B functions at xi (cell units),
// from the same a_i, b_i, c_i: da/dxi = -2 (fi + 1 - xi), db/dxi = 2 - 4 t,
// dc/dxi = 2 t with t = xi - fi.
void weight_grads_1d(double xi, double dN[4]) {
  const double fi = std::floor(xi);
  const double t = xi - fi;
  const double da = -2.0 * (fi + 1.0 - xi);
  const double db = 2.0 - 4.0 * t;
  const double dc = 2.0 * t;
  dN[0] = 0.25 * da;
  dN[1] = 0.25 * (da + db);
  dN[2] = 0.25 * (db + dc);
  dN[3] = 0.25 * dc;
}

bool inv3(const double A[9], double R[9]) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (det == 0.0 || !std::isfinite(det)) return false;
  const double id = 1.0 / det;
  R[0] = (A[4] * A[8] - A[5] * A[7]) * id;
  R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  R[3] = (A[5] * A[6] - A[3] * A[8]) * id;
  R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  R[6] = (A[3] * A[7] - A[4] * A[6]) * id;
  R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return true;
}

// The 64 background nodes a particle touches, their weights N_i(x_p) and
// offsets x_i - x_p, plus D_p and its inverse.  Positions are fixed for the
// whole contact step (Sec. 2.2), so this is built once per step.
struct Stencil {
  int32_t node[64];
  double w[64];
  double r[64][3];
  double D[9], Dinv[9];
};

struct Grid {
  std::unordered_map<Key, int32_t, KeyHash> index;
  std::vector<Key> keys;
  int32_t get(const Key& k) {
    auto it = index.find(k);
    if (it != index.end()) return it->second;
    const int32_t id = (int32_t)keys.size();
    index.emplace(k, id);
    keys.push_back(k);
    return id;
  }
};

void build_stencils(int64_t n, const double* x, double h, Grid& g, std::vector<Stencil>& st) {
  st.resize((size_t)n);
  for (int64_t p = 0; p < n; ++p) {
    Stencil& s = st[(size_t)p];
    double N[3][4];
    int64_t il[3];
    for (int d = 0; d < 3; ++d) weights_1d(x[3 * p + d] / h, &il[d], N[d]);
    int q = 0;
    for (int kz = 0; kz < 4; ++kz)
      for (int ky = 0; ky < 4; ++ky)
        for (int kx = 0; kx < 4; ++kx, ++q) {
          const Key key{il[0] - 1 + kx, il[1] - 1 + ky, il[2] - 1 + kz};
          s.node[q] = g.get(key);
          s.w[q] = N[0][kx] * N[1][ky] * N[2][kz];
          // x_i - x_p with x_i = h * (node index)
          s.r[q][0] = h * (double)key.i - x[3 * p + 0];
          s.r[q][1] = h * (double)key.j - x[3 * p + 1];
          s.r[q][2] = h * (double)key.k - x[3 * p + 2];
        }
    // D_p = sum_i N_i (x_i - x_p) (x) (x_i - x_p)   (Sec. 2.1.2)
    for (int a = 0; a < 9; ++a) s.D[a] = 0.0;
    for (int q2 = 0; q2 < 64; ++q2)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s.D[3 * a + b] += s.w[q2] * s.r[q2][a] * s.r[q2][b];
    inv3(s.D, s.Dinv);
  }
}

// eq. massToGrid
void grid_mass(int64_t n, const std::vector<Stencil>& st, const double* m, size_t G,
               std::vector<double>& mi) {
  mi.assign(G, 0.0);
  for (int64_t p = 0; p < n; ++p)
    for (int q = 0; q < 64; ++q) mi[(size_t)st[(size_t)p].node[q]] += st[(size_t)p].w[q] * m[p];
}

// eq. particleToGrid:  m_i v_i = sum_p N_i(x_p) m_p [ v_p + B_p D_p^{-1} (x_i - x_p) ]
// with B_p D_p^{-1} = C_p.  PIC drops the affine term.
void p2g_momentum(int64_t n, const std::vector<Stencil>& st, const double* m, const double* v,
                  const double* C, bool pic, size_t G, std::vector<double>& pi) {
  pi.assign(3 * G, 0.0);
  for (int64_t p = 0; p < n; ++p) {
    const Stencil& s = st[(size_t)p];
    for (int q = 0; q < 64; ++q) {
      double u[3];
      for (int a = 0; a < 3; ++a) {
        double aff = 0.0;
        if (!pic)
          for (int b = 0; b < 3; ++b) aff += C[9 * p + 3 * a + b] * s.r[q][b];
        u[a] = v[3 * p + a] + aff;
      }
      for (int a = 0; a < 3; ++a) pi[3 * (size_t)s.node[q] + a] += s.w[q] * m[p] * u[a];
    }
  }
}

// v_i = (m_i v_i) / m_i, and 0 where no mass reached the node.
void grid_velocity(size_t G, const std::vector<double>& mi, const std::vector<double>& pi,
                   std::vector<double>& vi) {
  vi.assign(3 * G, 0.0);
  for (size_t i = 0; i < G; ++i)
    if (mi[i] != 0.0)
      for (int a = 0; a < 3; ++a) vi[3 * i + a] = pi[3 * i + a] / mi[i];
}

// eq. gridToParticle and eq. scaledVelGrad; C_p = B_p D_p^{-1}.
void g2p(int64_t n, const std::vector<Stencil>& st, const std::vector<double>& vi, bool pic,
         const double* Cin, double* vout, double* Cout) {
  for (int64_t p = 0; p < n; ++p) {
    const Stencil& s = st[(size_t)p];
    double vh[3] = {0, 0, 0}, B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < 64; ++q) {
      const double* vq = &vi[3 * (size_t)s.node[q]];
      for (int a = 0; a < 3; ++a) {
        vh[a] += s.w[q] * vq[a];
        for (int b = 0; b < 3; ++b) B[3 * a + b] += s.w[q] * vq[a] * s.r[q][b];
      }
    }
    for (int a = 0; a < 3; ++a) vout[3 * p + a] = vh[a];
    if (pic) {
      // PIC carries no affine dofs: the C part passes through unchanged.
      for (int a = 0; a < 9; ++a) Cout[9 * p + a] = Cin[9 * p + a];
    } else {
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double c = 0.0;
          for (int k = 0; k < 3; ++k) c += B[3 * a + k] * s.Dinv[3 * k + b];
          Cout[9 * p + 3 * a + b] = c;
        }
    }
  }
}

// One application of the transfer operator H (Sec. 2.1.2): P2G then G2P.
void apply_H(int64_t n, const std::vector<Stencil>& st, const double* m,
             const std::vector<double>& mi, size_t G, bool pic, const double* v, const double* C,
             double* vout, double* Cout) {
  std::vector<double> pi, vi;
  p2g_momentum(n, st, m, v, C, pic, G, pi);
  grid_velocity(G, mi, pi, vi);
  g2p(n, st, vi, pic, C, vout, Cout);
}

// Sec. 2.4: undesirable part of a proposed velocity change, with the
// tangential part (I - n n) dv (the printed "dv n (x) n" is read as the
// tangential projection, the only reading for which the result is a cone
// projection) and the cone condition ||dv^t|| <= -mu dv.n.  A zero tangential
// part contributes nothing (0/0 read as 0).  Sec. 2.3 (flag): the whole
// change is undesirable if dv.n > 0, else nothing is.
void undesirable(const double dv[3], const double dC[9], const double nrm[3], double mu,
                 uint32_t flags, double dvu[3], double dCu[9]) {
  const double dn = dv[0] * nrm[0] + dv[1] * nrm[1] + dv[2] * nrm[2];
  if (flags & ORC_SEP23) {
    const bool sep = dn > 0.0;
    for (int a = 0; a < 3; ++a) dvu[a] = sep ? dv[a] : 0.0;
    for (int a = 0; a < 9; ++a) dCu[a] = sep ? dC[a] : 0.0;
    return;
  }
  if (dn <= 0.0) {
    double vt[3];
    for (int a = 0; a < 3; ++a) vt[a] = dv[a] - dn * nrm[a];
    const double nt = std::sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
    const double s = std::min(nt, -mu * dn);
    for (int a = 0; a < 3; ++a) dvu[a] = dv[a] - dn * nrm[a] - (nt > 0.0 ? s * vt[a] / nt : 0.0);
  } else {
    for (int a = 0; a < 3; ++a) dvu[a] = dv[a];
  }
  for (int a = 0; a < 9; ++a) dCu[a] = dC[a];
}

// Total linear and angular momentum of particles carrying {v_p, B_p}:
//   P = sum m v,   L = sum m [ x (x) v + eps_abc (B_p)_cb ]
// The spin term is what the grid sees: sum_i N_i (x_i - x_p) x (C_p (x_i - x_p))
// = eps_abc (C_p D_p)_cb.  B_p = C_p D_p with D_p from the weights.
void momentum(int64_t n, const std::vector<Stencil>* st, const double* x, const double* v,
              const double* C, const double* m, double h, double P[3], double L[3]) {
  for (int a = 0; a < 3; ++a) P[a] = L[a] = 0.0;
  for (int64_t p = 0; p < n; ++p) {
    const double* xp = x + 3 * p;
    const double* vp = v + 3 * p;
    double D[9];
    if (st) {
      for (int a = 0; a < 9; ++a) D[a] = (*st)[(size_t)p].D[a];
    } else {
      for (int a = 0; a < 9; ++a) D[a] = 0.0;
      D[0] = D[4] = D[8] = 0.5 * h * h;
    }
    double B[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += C[9 * p + 3 * a + k] * D[3 * k + b];
        B[3 * a + b] = s;
      }
    const double spin[3] = {B[3 * 2 + 1] - B[3 * 1 + 2], B[3 * 0 + 2] - B[3 * 2 + 0],
                            B[3 * 1 + 0] - B[3 * 0 + 1]};
    const double xv[3] = {xp[1] * vp[2] - xp[2] * vp[1], xp[2] * vp[0] - xp[0] * vp[2],
                          xp[0] * vp[1] - xp[1] * vp[0]};
    for (int a = 0; a < 3; ++a) {
      P[a] += m[p] * vp[a];
      L[a] += m[p] * (xv[a] + spin[a]);
    }
  }
}

}  // namespace

extern "C" {

// Flag values exported so the Python side does not duplicate them.
uint32_t oracle_flag_pic(void) { return ORC_PIC; }
uint32_t oracle_flag_sep23(void) { return ORC_SEP23; }

// App. B weights of the four nodes i-1..i+2 covering xi = x/h.
void oracle_weights(double xi, int64_t* ileft, double N[4]) { weights_1d(xi, ileft, N); }

// The undesirable part W of a proposed change {dv, dC} (Sec. 2.4 / 2.3).
void oracle_undesirable(const double* dv, const double* dC, const double* nrm, double mu,
                        uint32_t flags, double* dvu, double* dCu) {
  undesirable(dv, dC, nrm, mu, flags, dvu, dCu);
}

// Per-particle D_p (row-major 3x3) as computed from the weights.
int oracle_D(int64_t n, const double* x, double h, double* D) {
  if (n < 0 || !(h > 0.0)) return -1;
  Grid g;
  std::vector<Stencil> st;
  build_stencils(n, x, h, g, st);
  for (int64_t p = 0; p < n; ++p)
    for (int a = 0; a < 9; ++a) D[9 * p + a] = st[(size_t)p].D[a];
  return 0;
}

// P2G only: the grid nodes touched (integer coordinates), their mass and
// momentum.  Arrays must hold 64*n nodes.  Returns the node count.
int64_t oracle_p2g_grid(int64_t n, const double* x, const double* v, const double* C,
                        const double* m, double h, uint32_t flags, int64_t* node_ijk,
                        double* mass, double* mom) {
  if (n < 0 || !(h > 0.0)) return -1;
  Grid g;
  std::vector<Stencil> st;
  build_stencils(n, x, h, g, st);
  const size_t G = g.keys.size();
  std::vector<double> mi, pi;
  grid_mass(n, st, m, G, mi);
  p2g_momentum(n, st, m, v, C, (flags & ORC_PIC) != 0, G, pi);
  for (size_t i = 0; i < G; ++i) {
    node_ijk[3 * i + 0] = g.keys[i].i;
    node_ijk[3 * i + 1] = g.keys[i].j;
    node_ijk[3 * i + 2] = g.keys[i].k;
    mass[i] = mi[i];
    for (int a = 0; a < 3; ++a) mom[3 * i + a] = pi[3 * i + a];
  }
  return (int64_t)G;
}

// G2P only, from grid velocities given on listed nodes (nodes a particle
// touches that are not listed carry zero velocity).
int oracle_g2p_from_grid(int64_t n, const double* x, double h, uint32_t flags, int64_t G,
                         const int64_t* node_ijk, const double* vgrid, const double* Cin,
                         double* vout, double* Cout) {
  if (n < 0 || G < 0 || !(h > 0.0)) return -1;
  Grid g;
  for (int64_t i = 0; i < G; ++i) g.get(Key{node_ijk[3 * i], node_ijk[3 * i + 1], node_ijk[3 * i + 2]});
  std::vector<Stencil> st;
  build_stencils(n, x, h, g, st);
  std::vector<double> vi(3 * g.keys.size(), 0.0);
  for (int64_t i = 0; i < 3 * G; ++i) vi[(size_t)i] = vgrid[i];
  g2p(n, st, vi, (flags & ORC_PIC) != 0, Cin, vout, Cout);
  return 0;
}

// One application of H to {v, C}.
int oracle_apply_H(int64_t n, const double* x, const double* v, const double* C, const double* m,
                   double h, uint32_t flags, double* vout, double* Cout) {
  if (n < 0 || !(h > 0.0)) return -1;
  Grid g;
  std::vector<Stencil> st;
  build_stencils(n, x, h, g, st);
  const size_t G = g.keys.size();
  std::vector<double> mi;
  grid_mass(n, st, m, G, mi);
  apply_H(n, st, m, mi, G, (flags & ORC_PIC) != 0, v, C, vout, Cout);
  return 0;
}

// Momentum of a particle state (D_p computed from the weights).
int oracle_momentum(int64_t n, const double* x, const double* v, const double* C,
                    const double* m, double h, double* P, double* L) {
  if (n < 0 || !(h > 0.0)) return -1;
  Grid g;
  std::vector<Stencil> st;
  build_stencils(n, x, h, g, st);
  momentum(n, &st, x, v, C, m, h, P, L);
  return 0;
}

// The contact step: V_hat = V + G V + sum_{n=1..N} G W_n   (Sec. 2.3),
// W_{m+1} = undesirable(V_hat_m - V)                      (Sec. 2.4).
//
// x[n*3] positions; v[n*3], C[n*9] (row-major, C[3a+b] = dv_a/dx_b) the
// predicted generalized velocity; m[n] masses; nrm[n*3] outward normals
// (zero for interior nodes); body[n] in [0, n_bodies).  mu is the scalar
// friction coefficient; mu_pair (n_bodies^2, symmetric, may be NULL) gives a
// per-body-pair coefficient, blended per particle by the mass of the other
// bodies in its stencil (a reading; the paper has one scalar mu).
// stats (may be NULL) receives P_in[3], P_out[3], L_in[3], L_out[3] and the
// number of nodes touched by two or more bodies.
int oracle_contact_step(int64_t n, int32_t n_bodies, const int32_t* body, const double* x,
                        const double* v, const double* C, const double* m, const double* nrm,
                        double h, double mu, const double* mu_pair, int32_t n_iter,
                        uint32_t flags, double* v_out, double* C_out, double* stats) {
  if (n < 0 || n_bodies < 1 || !(h > 0.0) || n_iter < 0 || mu < 0.0) return -1;
  for (int64_t p = 0; p < n; ++p)
    if (body[p] < 0 || body[p] >= n_bodies || !(m[p] > 0.0)) return -1;
  const bool pic = (flags & ORC_PIC) != 0;
  Grid g;
  std::vector<Stencil> st;
  build_stencils(n, x, h, g, st);
  const size_t G = g.keys.size();
  std::vector<double> mi;
  grid_mass(n, st, m, G, mi);

  // Per-body node masses: which nodes more than one body touches, and the
  // per-particle friction coefficient when a pair table is given.
  std::vector<double> mb((size_t)n_bodies * G, 0.0);
  for (int64_t p = 0; p < n; ++p)
    for (int q = 0; q < 64; ++q)
      mb[(size_t)body[p] * G + (size_t)st[(size_t)p].node[q]] += st[(size_t)p].w[q] * m[p];
  int64_t multibody = 0;
  for (size_t i = 0; i < G; ++i) {
    int cnt = 0;
    for (int b = 0; b < n_bodies; ++b) cnt += mb[(size_t)b * G + i] > 0.0;
    multibody += cnt >= 2;
  }
  std::vector<double> mup((size_t)n, mu);
  if (mu_pair) {
    for (int64_t p = 0; p < n; ++p) {
      const int b = body[p];
      double num = 0.0, den = 0.0;
      for (int bo = 0; bo < n_bodies; ++bo) {
        if (bo == b) continue;
        double M = 0.0;  // mass of body bo seen through p's stencil
        for (int q = 0; q < 64; ++q) M += st[(size_t)p].w[q] * mb[(size_t)bo * G + st[(size_t)p].node[q]];
        num += mu_pair[b * n_bodies + bo] * M;
        den += M;
      }
      mup[(size_t)p] = den > 0.0 ? num / den : mu_pair[b * n_bodies + b];
    }
  }

  const size_t nv = 3 * (size_t)n, nc = 9 * (size_t)n;
  std::vector<double> Hv(nv), HC(nc), dv(nv), dC(nc), Wv(nv), WC(nc);
  // Delta_0 = H V - V
  apply_H(n, st, m, mi, G, pic, v, C, Hv.data(), HC.data());
  for (size_t k = 0; k < nv; ++k) dv[k] = Hv[k] - v[k];
  for (size_t k = 0; k < nc; ++k) dC[k] = HC[k] - C[k];
  for (int32_t it = 0; it < n_iter; ++it) {
    // W_{m+1} from the current proposed change
    for (int64_t p = 0; p < n; ++p)
      undesirable(&dv[3 * p], &dC[9 * p], &nrm[3 * p], mup[(size_t)p], flags, &Wv[3 * p],
                  &WC[9 * p]);
    // Delta_{m+1} = Delta_m + H W_{m+1} - W_{m+1}
    apply_H(n, st, m, mi, G, pic, Wv.data(), WC.data(), Hv.data(), HC.data());
    for (size_t k = 0; k < nv; ++k) dv[k] += Hv[k] - Wv[k];
    for (size_t k = 0; k < nc; ++k) dC[k] += HC[k] - WC[k];
  }
  for (size_t k = 0; k < nv; ++k) v_out[k] = v[k] + dv[k];
  for (size_t k = 0; k < nc; ++k) C_out[k] = C[k] + dC[k];
  if (stats) {
    momentum(n, &st, x, v, C, m, h, stats + 0, stats + 6);
    momentum(n, &st, x, v_out, C_out, m, h, stats + 3, stats + 9);
    stats[12] = (double)multibody;
  }
  return 0;
}

// 1-D transfers with linear hat functions (Sec. 3.1): nodes at x0 + h j,
// N_j(x) = max(0, 1 - |x - x_j| / h), D_p = sum_j N_j (x_j - x_p)^2,
// P2G m_j v_j = sum_p N_j m_p (v_p + B_p D_p^{-1} (x_j - x_p)),
// G2P v_p = sum_j N_j v_j, B_p = sum_j N_j v_j (x_j - x_p).
int oracle_apic1d_linear(int64_t n, const double* x, const double* v, const double* B,
                         const double* m, double h, double x0, double* vout, double* Bout) {
  if (n < 0 || !(h > 0.0)) return -1;
  std::unordered_map<int64_t, double> mj, pj;
  std::vector<int64_t> jl((size_t)n);
  std::vector<double> Dp((size_t)n);
  auto hat = [&](double xp, int64_t j) {
    const double xj = x0 + h * (double)j;
    return std::max(0.0, 1.0 - std::fabs(xp - xj) / h);
  };
  for (int64_t p = 0; p < n; ++p) {
    jl[(size_t)p] = (int64_t)std::floor((x[p] - x0) / h);
    double D = 0.0;
    for (int64_t j = jl[(size_t)p]; j <= jl[(size_t)p] + 1; ++j) {
      const double r = x0 + h * (double)j - x[p];
      D += hat(x[p], j) * r * r;
    }
    Dp[(size_t)p] = D;
  }
  for (int64_t p = 0; p < n; ++p)
    for (int64_t j = jl[(size_t)p]; j <= jl[(size_t)p] + 1; ++j) {
      const double N = hat(x[p], j);
      const double r = x0 + h * (double)j - x[p];
      const double aff = Dp[(size_t)p] > 0.0 ? B[p] / Dp[(size_t)p] * r : 0.0;
      mj[j] += N * m[p];
      pj[j] += N * m[p] * (v[p] + aff);
    }
  for (int64_t p = 0; p < n; ++p) {
    double vh = 0.0, bh = 0.0;
    for (int64_t j = jl[(size_t)p]; j <= jl[(size_t)p] + 1; ++j) {
      const double N = hat(x[p], j);
      const double r = x0 + h * (double)j - x[p];
      const double vj = mj[j] != 0.0 ? pj[j] / mj[j] : 0.0;
      vh += N * vj;
      bh += N * vj * r;
    }
    vout[p] = vh;
    Bout[p] = bh;
  }
  return 0;
}

// Node normals (Sec. 2.3, where the normal n_p of each particle is built):
// the outward normals of the boundary faces adjacent to a node, weighted by
// face area, summed and normalised.  Faces are triangles (a, b, c) wound
// counter-clockwise seen from outside, so that (b - a) x (c - a) points
// outward with length twice the area.  Nodes on no face, or whose weighted
// sum vanishes, get n = 0.  Returns -1 for an index outside [0, n).
int oracle_node_normals(int64_t n, const double* x, int64_t n_tri, const int32_t* tri, double* nrm) {
  if (n < 0 || n_tri < 0) return -1;
  std::vector<double> acc((size_t)(3 * n), 0.0);
  for (int64_t f = 0; f < n_tri; ++f) {
    const int32_t a = tri[3 * f], b = tri[3 * f + 1], c = tri[3 * f + 2];
    if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) return -1;
    double e1[3], e2[3], an[3];
    for (int k = 0; k < 3; ++k) {
      e1[k] = x[3 * b + k] - x[3 * a + k];
      e2[k] = x[3 * c + k] - x[3 * a + k];
    }
    // area times unit outward normal = half the cross product
    an[0] = 0.5 * (e1[1] * e2[2] - e1[2] * e2[1]);
    an[1] = 0.5 * (e1[2] * e2[0] - e1[0] * e2[2]);
    an[2] = 0.5 * (e1[0] * e2[1] - e1[1] * e2[0]);
    for (int32_t v : {a, b, c})
      for (int k = 0; k < 3; ++k) acc[(size_t)(3 * v + k)] += an[k];
  }
  for (int64_t p = 0; p < n; ++p) {
    const double* s = &acc[(size_t)(3 * p)];
    const double len = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    for (int k = 0; k < 3; ++k) nrm[3 * p + k] = len > 0.0 ? s[k] / len : 0.0;
  }
  return 0;
}

// Augury dynamics (Sec. 2.2): eq. apic_augury integrated with eq. Newmark,
// here with a linear-spring foreground (a stand-in for the paper's finite
// elements) plus uniform gravity.  The printed eq. Newmark has its half-step
// indices garbled; it is read as velocity Verlet (explicit Newmark,
// gamma = 1/2):
//   V^{n+1/2} = V^n + dt/2 A^n
//   x^{n+1}   = x^n + dt v^{n+1/2}
//   A^{n+1}   = {a(x^{n+1}), 0} + A_hat^{n+1}
//   V^{n+1}   = V^{n+1/2} + dt/2 A^{n+1}
// with eq. apic_accel A_hat = (H - I) V_bar / tau, V_bar = V_t + tau {a, 0},
// where V_t, the velocity at t^{n+1} before contact, is V^{n+1/2} + dt/2 {a, 0}
// (the mechanical part of the last half kick), and H is the contact step
// (the Sec. 2.3 series with the Sec. 2.4 projection) on normals built from
// the boundary triangles at x^{n+1}.  Fixed nodes (fixed[p] != 0) keep
// v = 0, C = 0, A = 0.  `init` first computes A^0 at x^0 with V_t = V^0.
// av[n*3], aC[n*9] carry A between calls.  energy (may be NULL) receives
// [kinetic 1/2 m |v|^2, spring energy, gravity energy -m g.x] after the run.
int oracle_augury_steps(int64_t n, int32_t n_bodies, const int32_t* body, double* x, double* v, double* C,
                        double* av, double* aC, const double* m, const uint8_t* fixed, int64_t n_springs,
                        const int32_t* springs, const double* rest, const double* k, const double* g,
                        int64_t n_tri, const int32_t* tri, double h, double mu, const double* mu_pair,
                        int32_t n_iter, uint32_t flags, double dt, double tau, int32_t n_steps, int32_t init,
                        double* energy) {
  if (n <= 0 || !(dt > 0.0) || !(tau > 0.0) || n_steps < 0) return -1;
  for (int64_t s = 0; s < n_springs; ++s)
    if (springs[2 * s] < 0 || springs[2 * s] >= n || springs[2 * s + 1] < 0 || springs[2 * s + 1] >= n) return -1;
  std::vector<double> am((size_t)(3 * n)), nrm((size_t)(3 * n), 0.0), vbar((size_t)(3 * n)),
      vhat((size_t)(3 * n)), Chat((size_t)(9 * n));
  auto is_fixed = [&](int64_t p) { return fixed && fixed[p]; };
  // a(x): spring forces / m + g
  auto mechanical = [&]() {
    for (int64_t p = 0; p < n; ++p)
      for (int c = 0; c < 3; ++c) am[(size_t)(3 * p + c)] = 0.0;
    for (int64_t s = 0; s < n_springs; ++s) {
      const int32_t i = springs[2 * s], j = springs[2 * s + 1];
      double d[3], len2 = 0.0;
      for (int c = 0; c < 3; ++c) {
        d[c] = x[3 * j + c] - x[3 * i + c];
        len2 += d[c] * d[c];
      }
      const double len = std::sqrt(len2);
      if (!(len > 0.0)) continue;
      const double f = k[s] * (len - rest[s]) / len;  // pulls i toward j when stretched
      for (int c = 0; c < 3; ++c) {
        am[(size_t)(3 * i + c)] += f * d[c];
        am[(size_t)(3 * j + c)] -= f * d[c];
      }
    }
    for (int64_t p = 0; p < n; ++p)
      for (int c = 0; c < 3; ++c) am[(size_t)(3 * p + c)] = am[(size_t)(3 * p + c)] / m[p] + (g ? g[c] : 0.0);
  };
  // A = {a, 0} + (H - I) V_bar / tau with V_bar = (v_t + tau a, C)
  auto accelerate = [&](const double* vt) -> int {
    if (n_tri > 0 && oracle_node_normals(n, x, n_tri, tri, nrm.data()) != 0) return -1;
    for (int64_t i = 0; i < 3 * n; ++i) vbar[(size_t)i] = vt[i] + tau * am[(size_t)i];
    if (oracle_contact_step(n, n_bodies, body, x, vbar.data(), C, m, nrm.data(), h, mu, mu_pair, n_iter, flags,
                            vhat.data(), Chat.data(), nullptr) != 0)
      return -1;
    for (int64_t p = 0; p < n; ++p) {
      for (int c = 0; c < 3; ++c) {
        const size_t i = (size_t)(3 * p + c);
        av[i] = is_fixed(p) ? 0.0 : am[i] + (vhat[i] - vbar[i]) / tau;
      }
      for (int c = 0; c < 9; ++c) {
        const size_t i = (size_t)(9 * p + c);
        aC[i] = is_fixed(p) ? 0.0 : (Chat[i] - C[i]) / tau;
      }
    }
    return 0;
  };
  std::vector<double> vt((size_t)(3 * n));
  if (init) {
    mechanical();
    if (accelerate(v) != 0) return -1;
  }
  for (int32_t step = 0; step < n_steps; ++step) {
    for (int64_t p = 0; p < n; ++p) {  // V^{n+1/2}, x^{n+1}
      for (int c = 0; c < 3; ++c) v[3 * p + c] = is_fixed(p) ? 0.0 : v[3 * p + c] + 0.5 * dt * av[3 * p + c];
      for (int c = 0; c < 9; ++c) C[9 * p + c] = is_fixed(p) ? 0.0 : C[9 * p + c] + 0.5 * dt * aC[9 * p + c];
      for (int c = 0; c < 3; ++c) x[3 * p + c] += dt * v[3 * p + c];
    }
    mechanical();  // a(x^{n+1})
    for (int64_t i = 0; i < 3 * n; ++i) vt[(size_t)i] = v[i] + 0.5 * dt * am[(size_t)i];
    if (accelerate(vt.data()) != 0) return -1;
    for (int64_t p = 0; p < n; ++p) {  // V^{n+1}
      for (int c = 0; c < 3; ++c) v[3 * p + c] += 0.5 * dt * av[3 * p + c];
      for (int c = 0; c < 9; ++c) C[9 * p + c] += 0.5 * dt * aC[9 * p + c];
    }
  }
  if (energy) {
    double kin = 0.0, spr = 0.0, grav = 0.0;
    for (int64_t p = 0; p < n; ++p)
      for (int c = 0; c < 3; ++c) {
        kin += 0.5 * m[p] * v[3 * p + c] * v[3 * p + c];
        grav -= m[p] * (g ? g[c] : 0.0) * x[3 * p + c];
      }
    for (int64_t s = 0; s < n_springs; ++s) {
      const int32_t i = springs[2 * s], j = springs[2 * s + 1];
      double len2 = 0.0;
      for (int c = 0; c < 3; ++c) len2 += (x[3 * j + c] - x[3 * i + c]) * (x[3 * j + c] - x[3 * i + c]);
      const double e = std::sqrt(len2) - rest[s];
      spr += 0.5 * k[s] * e * e;
    }
    energy[0] = kin;
    energy[1] = spr;
    energy[2] = grav;
  }
  return 0;
}

// Derivatives of the App. B weights with respect to xi = x/h.
void oracle_weight_grads(double xi, double dN[4]) { weight_grads_1d(xi, dN); }

// Normals from the bodies' grid mass (for callers with no surface mesh; the
// paper's normals come from the FE surface, Sec. 2.3, so this is a reading):
// for particle p of body b, rho_p = sum_i N_i(x_p) m_{b,i} and
// g_p = sum_i dN_i/dxi(x_p) m_{b,i}, the body's grid mass (eq. massToGrid
// over body b alone) interpolated back and its gradient in cell units.  The
// mass falls off outward, so n_p = -g_p / |g_p| where |g_p| > threshold *
// rho_p, and n_p = 0 inside the body (a uniform mass field has g_p = 0, the
// App. B weights summing to one).  ratio[p] = |g_p| / rho_p (may be NULL).
int oracle_mass_normals(int64_t n, int32_t n_bodies, const int32_t* body, const double* x, const double* m,
                        double h, double threshold, double* nrm, double* ratio) {
  if (n < 0 || n_bodies < 1 || !(h > 0.0) || !(threshold >= 0.0)) return -1;
  for (int64_t p = 0; p < n; ++p)
    if (body[p] < 0 || body[p] >= n_bodies || !(m[p] > 0.0)) return -1;
  Grid g;
  std::vector<Stencil> st;
  build_stencils(n, x, h, g, st);
  const size_t G = g.keys.size();
  // per-body node masses
  std::vector<double> mb((size_t)n_bodies * G, 0.0);
  for (int64_t p = 0; p < n; ++p)
    for (int q = 0; q < 64; ++q)
      mb[(size_t)body[p] * G + (size_t)st[(size_t)p].node[q]] += st[(size_t)p].w[q] * m[p];
  for (int64_t p = 0; p < n; ++p) {
    double N[3][4], dN[3][4];
    int64_t il[3];
    for (int d = 0; d < 3; ++d) {
      weights_1d(x[3 * p + d] / h, &il[d], N[d]);
      weight_grads_1d(x[3 * p + d] / h, dN[d]);
    }
    const double* mbb = &mb[(size_t)body[p] * G];
    double rho = 0.0, gr[3] = {0.0, 0.0, 0.0};
    int q = 0;
    for (int kz = 0; kz < 4; ++kz)
      for (int ky = 0; ky < 4; ++ky)
        for (int kx = 0; kx < 4; ++kx, ++q) {
          const double mi = mbb[(size_t)st[(size_t)p].node[q]];
          rho += N[0][kx] * N[1][ky] * N[2][kz] * mi;
          gr[0] += dN[0][kx] * N[1][ky] * N[2][kz] * mi;
          gr[1] += N[0][kx] * dN[1][ky] * N[2][kz] * mi;
          gr[2] += N[0][kx] * N[1][ky] * dN[2][kz] * mi;
        }
    const double len = std::sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    const double r = rho > 0.0 ? len / rho : 0.0;
    if (ratio) ratio[p] = r;
    for (int a = 0; a < 3; ++a) nrm[3 * p + a] = (r > threshold && len > 0.0) ? -gr[a] / len : 0.0;
  }
  return 0;
}

}  // extern "C"
