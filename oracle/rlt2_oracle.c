/*
 * CPU oracle for RLT2 Lagrangian dual ascent on the QAP (Date & Nagi,
 * "RLT2-based Parallel Algorithms for Solving Large Quadratic Assignment
 * Problems on Graphics Processing Unit Clusters").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, deliberately obvious
 * restatement of the method in FP64.  It is used by the test-suite, by the
 * package smoke check and by the benchmark's CPU-baseline leg; nothing on the
 * product path links, loads or calls it.  It shares no code with the CUDA
 * library.  Build flags: -O2 -ffp-contract=off: the compiler contracts
 * nothing, so every + and * below is one IEEE round-to-nearest operation and
 * a fused multiply-add happens only where the code calls C99 fma() (the z
 * move's regrouped forms, which the paper's formulas leave the order of).
 *
 * Notation follows the paper (Section 2.3):
 *   n facilities/locations, b (n x n), C_ijpq = f_ij d_pq (RLT1, Eq. 2.1),
 *   D_ijkpqr (RLT2, Eq. 2.6) = 0 for the QAP, multiplier-adjusted costs
 *   b', C^ = C - u, D^ = D - v (Section 3.3: the multipliers live inside the
 *   costs, there is no separate multiplier array).
 *   Z-LAP(i,j,p,q): rows k != i,j, cols r != p,q, cost D^_ijkpqr -> Theta, xi, psi
 *   Y-LAP(i,p):     rows j != i,   cols q != p,   cost C^_ijpq + Theta_ijpq -> Delta, gamma, delta
 *   X-LAP:          rows i,        cols p,        cost b'_ip + Delta_ip -> LB, alpha, beta
 *
 * Array layouts (shared by contract with the CUDA library, not by code):
 *   compressed index: j' = j - (j > i); k' = k - (k > i) - (k > j) (same for
 *   locations).  Tile t(i,p,j',q') = ((i*n + p)*(n-1) + j')*(n-1) + q'.
 *   C^[t], Theta[t], pi_y[t]; D^[t*m*m + k'*m + r'] with m = n-2;
 *   xi[t*m + k'], psi[t*m + r']; gamma/delta[(i*n+p)*(n-1) + j'/q'];
 *   Delta[i*n+p], pi_x[i*n+p], alpha[i], beta[p].
 *
 * Readings of points the paper leaves open:
 *   - state is (b', C^, D^); Theta and Delta are rebuilt every iteration
 *     (Algorithm 1's "C' <- C' + Theta" is read as a temporary, S1 variant);
 *   - all reduced costs come from one snapshot before any cost moves (Jacobi);
 *   - LAP duals: raw (this Hungarian's own) or canonical (pointwise-maximal
 *     row duals with u_0 = 0 among all optimal duals; unique);
 *   - per z entry a=(i,j,k,p,q,r), s(a) = fma(kz, pi_z(a), cy*pi_y(ijpq) + cx*pi_x(ip)),
 *     cy = ky/(n-2), cx = kx/((n-1)(n-2))  (Eq. 2.20, 2.22, 2.23 combined as
 *     in the proof of Theorem 1), and
 *     D^'(a) = (D^(a) - s(a)) + sum over the five partners b of phi(b->a)*s(b),
 *     the partner terms added one fused multiply-add (C99 fma) at a time; with
 *     all phi equal, D^'(a) = fma(phi, S - s(a), D^(a) - s(a)), S = sum of the
 *     class's six s in member order; with all phi equal and kz = 1 (the
 *     default) the same formula is regrouped as
 *     s(a) = (D^ - xi_k') - (psi_r' - ty), D^'(a) = fma(-(1+phi), s, fma(phi, S, D^));
 *   - an LAP optimum is summed as a pairwise tree;
 *   - y move (Eq. 2.21): C^'_ijpq = (C^_ijpq - phi_y*pi_y(ijpq)) + phi_y*pi_y(jiqp).
 * Variants (Section 3.4):
 *   - F: the LAPs run on the incremental costs of Psi_2 (Eq. 3.6): what is left
 *     of each reduced cost after the step plus the inflow; the bound is the
 *     previous bound plus the X-LAP value (Eq. 3.7).  With the y move of
 *     Eq. 2.21 the new y cost is (1 - ky - phi_y) pi_y(ijpq) + phi_y pi_y(jiqp);
 *   - two-phase Z solve: S_B = {pi_z <= tol (1 + |xi| + |psi|)} stands for
 *     "zero slack" (the paper's pi(z) = 0 after rounding); the S_N slack sum is
 *     shared as sum * (1/|S_B|);
 *   - Type 4 rule (Section 2.3 rule 4, Section 5): the amounts per coefficient
 *     are the printed ones (kappa_i nu / n per b, kappa_i nu / (n(n-1)(n-2)) per
 *     z); acceptance compares kappa^lb * nu with -ln(u) * T (u <= exp(-kappa^lb
 *     nu / T), the energy in the bound's units so that T = 4% of the upper
 *     bound is commensurate); the random fractions and -ln(u) are inputs;
 *   - half-Z scheme (Section 5): lower-order members keep cost 0 (their
 *     Z-LAPs are skipped); the y move of Eq. 2.21 runs with phi_y = 1/2 (the
 *     updated slack split equally between y_ijpq and y_jiqp); only the three
 *     upper members pool (kz pi_z + cy * [upper y slack after the y move] +
 *     cx pi_x) and share (1/2 to each other upper member); the x slack of the
 *     lower rows (i > j) moves on the y level, kx pi_x(ip)/(n-1) from y_ijpq
 *     to its mirror, so every Y-LAP row passes its share of pi_x on.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1

/* ------------------------------------------------------------------------ */
/* Linear assignment: shortest-augmenting-path Hungarian (primal-dual).      */
/* The paper solves every LAP with a Hungarian method (Section 3.2); this is  */
/* the textbook Dijkstra-based form with Jonker-Volgenant dual updates.       */
/* Reduced cost pi(r,c) = (c_rc - u_r) - v_c >= 0; matched edges have 0.      */
/* Ties always go to the lowest index; relaxations use strict '<'.            */
/* ------------------------------------------------------------------------ */
int or_lap(int m, const double* c, const double* u0, double* value, double* u, double* v,
           int* row_to_col, int* n_aug, long long* n_relax) {
  if (m <= 0) {
    if (value) *value = 0.0;
    if (n_aug) *n_aug = 0;
    if (n_relax) *n_relax = 0;
    return OR_OK;
  }
  int* col_to_row = (int*)malloc(sizeof(int) * m);
  int* argrow = (int*)malloc(sizeof(int) * m);
  int* pred = (int*)malloc(sizeof(int) * m);
  char* scanned = (char*)malloc(m);
  double* d = (double*)malloc(sizeof(double) * m);
  int aug = 0;
  long long relax = 0;

  /* start duals: u = u0 (or 0), v_c = min_r (c_rc - u_r) */
  for (int r = 0; r < m; r++) {
    u[r] = u0 ? u0[r] : 0.0;
    row_to_col[r] = -1;
  }
  for (int col = 0; col < m; col++) {
    double best = 0.0;
    int arg = -1;
    for (int r = 0; r < m; r++) {
      double x = c[r * m + col] - u[r];
      if (arg < 0 || x < best) {
        best = x;
        arg = r;
      }
    }
    v[col] = best;
    argrow[col] = arg;
    col_to_row[col] = -1;
  }
  /* greedy pass: column col takes its argmin row if that row is still free */
  for (int col = 0; col < m; col++) {
    int r = argrow[col];
    if (row_to_col[r] < 0) {
      row_to_col[r] = col;
      col_to_row[col] = r;
    }
  }
  /* one Dijkstra search per free row, rows in increasing order */
  for (int i = 0; i < m; i++) {
    if (row_to_col[i] >= 0) continue;
    aug++;
    for (int col = 0; col < m; col++) {
      d[col] = (c[i * m + col] - u[i]) - v[col];
      pred[col] = i;
      scanned[col] = 0;
    }
    relax += m;
    int sink = -1;
    double dlast = 0.0;
    for (;;) {
      int cs = -1;
      double dm = 0.0;
      for (int col = 0; col < m; col++) {
        if (scanned[col]) continue;
        if (cs < 0 || d[col] < dm) {
          cs = col;
          dm = d[col];
        }
      }
      scanned[cs] = 1;
      if (col_to_row[cs] < 0) {
        sink = cs;
        dlast = dm;
        break;
      }
      int r = col_to_row[cs];
      for (int col = 0; col < m; col++) {
        if (scanned[col]) continue;
        double nd = dm + ((c[r * m + col] - u[r]) - v[col]);
        relax++;
        if (nd < d[col]) {
          d[col] = nd;
          pred[col] = r;
        }
      }
    }
    /* dual update on the scanned columns */
    for (int col = 0; col < m; col++)
      if (scanned[col]) v[col] = v[col] + (d[col] - dlast);
    /* augment along the predecessor chain back to row i */
    int col = sink;
    for (;;) {
      int r = pred[col];
      int nxt = row_to_col[r];
      col_to_row[col] = r;
      row_to_col[r] = col;
      if (r == i) break;
      col = nxt;
    }
    /* row duals of matched rows from the tight matched edges */
    for (int r = 0; r < m; r++)
      if (row_to_col[r] >= 0) u[r] = c[r * m + row_to_col[r]] - v[row_to_col[r]];
  }
  /* optimum: pairwise tree sum over P = next power of two >= m leaves (rows
   * beyond m are empty), adding s[i] + s[i + h] for h = P/2, ..., 1 */
  double leaf[64];
  int P = 1;
  while (P < m) P <<= 1;
  for (int r = 0; r < P; r++) leaf[r] = r < m ? c[r * m + row_to_col[r]] : 0.0;
  for (int h = P / 2; h >= 1; h /= 2)
    for (int r = 0; r < h; r++) leaf[r] = leaf[r] + leaf[r + h];
  if (value) *value = leaf[0];
  if (n_aug) *n_aug = aug;
  if (n_relax) *n_relax = relax;
  free(col_to_row);
  free(argrow);
  free(pred);
  free(scanned);
  free(d);
  return OR_OK;
}

/* Canonical optimal dual of an LAP, given an optimal assignment sigma.
 * All optimal duals satisfy u_r - u_r' <= c[r][sigma(r')] - c[r'][sigma(r')]
 * (eliminate v through the tight matched edges).  With u_0 = 0 the pointwise
 * largest solution is the shortest-path distance from row 0 in the graph with
 * arcs r' -> r of that weight; computed here by plain Bellman-Ford.  The set of
 * optimal duals does not depend on which optimal sigma was found, so neither
 * does this dual.  v_c = c[sigma^-1(c)][c] - u[sigma^-1(c)]. */
void or_lap_canonical(int m, const double* c, const int* row_to_col, double* u_out, double* v_out) {
  if (m <= 0) return;
  char* reached = (char*)calloc(m, 1);
  u_out[0] = 0.0;
  reached[0] = 1;
  for (int r = 1; r < m; r++) u_out[r] = 0.0;
  for (int round = 0; round < m - 1; round++) {
    int changed = 0;
    for (int rp = 0; rp < m; rp++) {
      if (!reached[rp]) continue;
      int sp = row_to_col[rp];
      for (int r = 1; r < m; r++) {
        if (r == rp) continue;
        double w = c[r * m + sp] - c[rp * m + sp];
        double nd = u_out[rp] + w;
        if (!reached[r] || nd < u_out[r]) {
          u_out[r] = nd;
          reached[r] = 1;
          changed = 1;
        }
      }
    }
    if (!changed) break;
  }
  for (int r = 0; r < m; r++) v_out[row_to_col[r]] = c[r * m + row_to_col[r]] - u_out[r];
  free(reached);
}

/* Brute-force LAP over all m! permutations (m <= 9): pins or_lap. */
static void lap_brute_rec(int m, const double* c, int r, int* perm, char* used, double acc, double* best,
                          int* bestp) {
  if (r == m) {
    if (acc < *best) {
      *best = acc;
      memcpy(bestp, perm, sizeof(int) * m);
    }
    return;
  }
  for (int col = 0; col < m; col++) {
    if (used[col]) continue;
    used[col] = 1;
    perm[r] = col;
    lap_brute_rec(m, c, r + 1, perm, used, acc + c[r * m + col], best, bestp);
    used[col] = 0;
  }
}
double or_lap_brute(int m, const double* c, int* best_perm) {
  int perm[16];
  char used[16] = {0};
  int bp[16];
  double best = INFINITY;
  if (m <= 0 || m > 10) return NAN;
  lap_brute_rec(m, c, 0, perm, used, 0.0, &best, bp);
  if (best_perm) memcpy(best_perm, bp, sizeof(int) * m);
  return best;
}

/* QAP objective of a permutation (Eq. 1.1): sum b_i,perm(i) + sum f_ij d_perm(i)perm(j). */
double or_qap_cost(int n, const double* F, const double* D, const double* B, const int* perm) {
  double s = 0.0;
  for (int i = 0; i < n; i++) {
    if (B) s += B[i * n + perm[i]];
    for (int j = 0; j < n; j++) s += F[i * n + j] * D[perm[i] * n + perm[j]];
  }
  return s;
}

/* Brute-force QAP optimum over all n! permutations (Heap's algorithm), n <= 11. */
double or_qap_brute(int n, const double* F, const double* D, const double* B, int* best_perm) {
  int perm[16], cnt[16];
  if (n <= 0 || n > 11) return NAN;
  for (int i = 0; i < n; i++) {
    perm[i] = i;
    cnt[i] = 0;
  }
  double best = or_qap_cost(n, F, D, B, perm);
  if (best_perm) memcpy(best_perm, perm, sizeof(int) * n);
  int i = 1;
  while (i < n) {
    if (cnt[i] < i) {
      int k = (i % 2 == 0) ? 0 : cnt[i];
      int tmp = perm[k];
      perm[k] = perm[i];
      perm[i] = tmp;
      double s = or_qap_cost(n, F, D, B, perm);
      if (s < best) {
        best = s;
        if (best_perm) memcpy(best_perm, perm, sizeof(int) * n);
      }
      cnt[i]++;
      i = 1;
    } else {
      cnt[i] = 0;
      i++;
    }
  }
  return best;
}

/* ------------------------------------------------------------------------ */
/* Index helpers                                                              */
/* ------------------------------------------------------------------------ */
static inline int cmp1(int j, int i) { return j - (j > i); }              /* j' of j != i */
static inline int cmp2(int k, int i, int j) { return k - (k > i) - (k > j); } /* k' of k != i,j */
static inline long long tile_of(int n, int i, int p, int j, int q) {
  return (((long long)i * n + p) * (n - 1) + cmp1(j, i)) * (n - 1) + cmp1(q, p);
}
long long or_num_tiles(int n) { return (long long)n * n * (n - 1) * (n - 1); }
long long or_num_z(int n) { return or_num_tiles(n) * (n - 2) * (n - 2); }

/* ------------------------------------------------------------------------ */
/* Setup (Eq. 1.1, 2.1, 2.6; partial assignment = fixed facilities of a       */
/* branch-and-bound node, Section 4).  Free facilities and free locations are */
/* renumbered in increasing order.  With a partial assignment phi on A:       */
/*   b'_ip = b_ip + f_ii d_pp + sum_{a in A} (f_ia d_{p,phi a} + f_ai d_{phi a,p})  */
/*   const = sum_{a in A} b_{a,phi a} + sum_{a,a' in A} f_aa' d_{phi a,phi a'} */
/*   C^_ijpq = f_ij d_pq (i != j, p != q), D^ = 0.                           */
/* ------------------------------------------------------------------------ */
int or_setup(int n, const double* F, const double* D, const double* B, const int* partial, int* n_res_out,
             double* cst_out, double* bprime, double* Chat, double* Dhat) {
  int fac[64], loc[64];
  int nf = 0, nl = 0;
  char locused[64] = {0};
  if (n < 1 || n > 64) return OR_EINVAL;
  for (int i = 0; i < n; i++) {
    if (partial && partial[i] >= 0) {
      if (partial[i] >= n || locused[partial[i]]) return OR_EINVAL;
      locused[partial[i]] = 1;
    }
  }
  for (int i = 0; i < n; i++)
    if (!partial || partial[i] < 0) fac[nf++] = i;
  for (int p = 0; p < n; p++)
    if (!locused[p]) loc[nl++] = p;
  if (nf != nl) return OR_EINVAL;
  int nr = nf;
  if (n_res_out) *n_res_out = nr;
  double cst = 0.0;
  if (partial) {
    for (int a = 0; a < n; a++) {
      if (partial[a] < 0) continue;
      if (B) cst += B[a * n + partial[a]];
      for (int a2 = 0; a2 < n; a2++) {
        if (partial[a2] < 0) continue;
        cst += F[a * n + a2] * D[partial[a] * n + partial[a2]];
      }
    }
  }
  if (cst_out) *cst_out = cst;
  for (int ii = 0; ii < nr; ii++) {
    for (int pp = 0; pp < nr; pp++) {
      int i = fac[ii], p = loc[pp];
      double s = (B ? B[i * n + p] : 0.0) + F[i * n + i] * D[p * n + p];
      if (partial) {
        for (int a = 0; a < n; a++) {
          if (partial[a] < 0) continue;
          s += F[i * n + a] * D[p * n + partial[a]] + F[a * n + i] * D[partial[a] * n + p];
        }
      }
      bprime[ii * nr + pp] = s;
    }
  }
  if (nr >= 2 && Chat) {
    for (int ii = 0; ii < nr; ii++)
      for (int jj = 0; jj < nr; jj++) {
        if (jj == ii) continue;
        for (int pp = 0; pp < nr; pp++)
          for (int qq = 0; qq < nr; qq++) {
            if (qq == pp) continue;
            Chat[tile_of(nr, ii, pp, jj, qq)] = F[fac[ii] * n + fac[jj]] * D[loc[pp] * n + loc[qq]];
          }
      }
  }
  if (nr >= 3 && Dhat) memset(Dhat, 0, sizeof(double) * (size_t)or_num_z(nr));
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Stages of one iteration (Algorithm 1, steps 3-5; Figure 1)                 */
/* ------------------------------------------------------------------------ */
static void solve_one(int m, const double* cost, const double* u0, int dual_mode, double* value, double* u,
                      double* v, int* perm, int* aug, long long* relax) {
  or_lap(m, cost, u0, value, u, v, perm, aug, relax);
  if (dual_mode == 1) {
    double* uc = (double*)malloc(sizeof(double) * m);
    double* vc = (double*)malloc(sizeof(double) * m);
    or_lap_canonical(m, cost, perm, uc, vc);
    memcpy(u, uc, sizeof(double) * m);
    memcpy(v, vc, sizeof(double) * m);
    free(uc);
    free(vc);
  }
}

/* Z stage: n^2 (n-1)^2 LAPs of size n-2 over the tiles of D^.  u0 (nullable)
 * holds starting row duals per tile (warm start). */
void or_stage_z(int n, int dual_mode, const double* Dhat, const double* u0, double* Theta, double* xi, double* psi,
                long long* naug, long long* nrelax, int nthreads) {
  long long T = or_num_tiles(n);
  int m = n - 2;
  long long aug_tot = 0, relax_tot = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1) reduction(+ : aug_tot, relax_tot)
#endif
  for (long long t = 0; t < T; t++) {
    int perm[64];
    int aug;
    long long relax;
    solve_one(m, Dhat + t * m * m, u0 ? u0 + t * m : NULL, dual_mode, &Theta[t], xi + t * m, psi + t * m, perm,
              &aug, &relax);
    aug_tot += aug;
    relax_tot += relax;
  }
  if (naug) *naug = aug_tot;
  if (nrelax) *nrelax = relax_tot;
  (void)nthreads;
}

/* Y stage: n^2 LAPs of size n-1 with cost C^ + Theta (Figure 1, second stage). */
void or_stage_y(int n, int dual_mode, const double* Chat, const double* Theta, const double* u0y, double* Delta,
                double* gamma, double* delta, long long* naug, long long* nrelax) {
  int m = n - 1;
  double* cost = (double*)malloc(sizeof(double) * m * m);
  long long aug_tot = 0, relax_tot = 0;
  for (int i = 0; i < n; i++)
    for (int p = 0; p < n; p++) {
      long long base = ((long long)i * n + p) * m * m;
      for (int e = 0; e < m * m; e++) cost[e] = Chat[base + e] + Theta[base + e];
      int perm[64];
      int aug;
      long long relax;
      solve_one(m, cost, u0y ? u0y + (i * n + p) * m : NULL, dual_mode, &Delta[i * n + p], gamma + (i * n + p) * m,
                delta + (i * n + p) * m,
                perm, &aug, &relax);
      aug_tot += aug;
      relax_tot += relax;
    }
  free(cost);
  if (naug) *naug = aug_tot;
  if (nrelax) *nrelax = relax_tot;
}

/* X stage: one LAP of size n with cost b' + Delta; its value is the bound. */
void or_stage_x(int n, int dual_mode, const double* bprime, const double* Delta, const double* u0x, double* lb,
                double* alpha, double* beta, int* xperm, long long* naug, long long* nrelax) {
  double* cost = (double*)malloc(sizeof(double) * n * n);
  for (int e = 0; e < n * n; e++) cost[e] = bprime[e] + Delta[e];
  int aug;
  long long relax;
  solve_one(n, cost, u0x, dual_mode, lb, alpha, beta, xperm, &aug, &relax);
  free(cost);
  if (naug) *naug = aug;
  if (nrelax) *nrelax = relax;
}

/* Reduced costs (Eq. 2.19 and the constraints of DLRLT2, Eq. 2.13-2.15):
 * pi_x(ip) = ((b'_ip + Delta_ip) - alpha_i) - beta_p
 * pi_y(t)  = ((C^_t + Theta_t) - gamma_ip[j']) - delta_ip[q']      */
void or_reduced_xy(int n, const double* bprime, const double* Delta, const double* alpha, const double* beta,
                   const double* Chat, const double* Theta, const double* gamma, const double* delta, double* pix,
                   double* piy) {
  int m = n - 1;
  for (int i = 0; i < n; i++)
    for (int p = 0; p < n; p++) pix[i * n + p] = ((bprime[i * n + p] + Delta[i * n + p]) - alpha[i]) - beta[p];
  for (int i = 0; i < n; i++)
    for (int p = 0; p < n; p++)
      for (int jp = 0; jp < m; jp++)
        for (int qp = 0; qp < m; qp++) {
          long long t = (((long long)i * n + p) * m + jp) * m + qp;
          piy[t] = ((Chat[t] + Theta[t]) - gamma[(i * n + p) * m + jp]) - delta[(i * n + p) * m + qp];
        }
}

/* pi_z of one entry: (D^ - xi_k') - psi_r'. */
static inline double piz_at(int n, const double* Dhat, const double* xi, const double* psi, int i, int j, int k, int p,
                            int q, int r) {
  int m = n - 2;
  long long t = tile_of(n, i, p, j, q);
  int kk = cmp2(k, i, j), rr = cmp2(r, p, q);
  return (Dhat[t * m * m + kk * m + rr] - xi[t * m + kk]) - psi[t * m + rr];
}
static inline long long zidx(int n, int i, int j, int k, int p, int q, int r) {
  int m = n - 2;
  return tile_of(n, i, p, j, q) * m * m + cmp2(k, i, j) * m + cmp2(r, p, q);
}

/* z redistribution (Types 1-3 combined, Eq. 2.20, 2.22, 2.23 and Eq. 2.25 in
 * the proof of Theorem 1), applied to D^ in place (Section 3.3).
 * prm = {kz, ky, kx, phi_y, phi_1..phi_5}.  The member a=(i,j,k,p,q,r) gives
 * phi_l * s(a) to its l-th partner, partners listed as in Eq. 2.20:
 *   1:(i,k,j,p,r,q) 2:(j,i,k,q,p,r) 3:(j,k,i,q,r,p) 4:(k,i,j,r,p,q) 5:(k,j,i,r,q,p).
 * Seen from the receiver a, the partners b1..b5 (same list) give it
 * phi_1, phi_2, phi_4, phi_3, phi_5 respectively (the two 3-cycles are each
 * other's inverse; the swaps are their own inverse). */
/* variant 0 (S): D^'(a) = (D^(a) - s(a)) + inflow.
 * variant 1 (F, Section 3.4 and the constraint set Psi_2 of Eq. 3.6): the z
 * cost is the incremental one, D^ holds the costs whose LAPs were just solved,
 * and the new incremental cost is what remains of the slack plus the inflow:
 * D^'(a) = fma(-kz, pi_z(a), pi_z(a)) [- sa(ip)] + inflow, i.e. (1-kz) pi_z
 * + Omega of Eq. 3.5 (the y and x parts of the pool leave the y and x costs).
 * sa (nullable, n*n): the Type 4 amount per (first facility, first location)
 * (Section 2.3, rule 4), added to every pool and, in F, taken from the z cost.
 * form 0 picks the regrouped branches where they apply (equal phi; equal phi
 * with kz = 1 in S); form 1 always takes the general branch, which adds the
 * five partner terms one at a time exactly as Eq. 2.20 lists them and is the
 * plain definition the regrouped branches are tested against. */
void or_redistribute_z_form(int n, const double* prm, int variant, const double* sa, int form, double* Dhat,
                            const double* xi, const double* psi, const double* piy, const double* pix, int nthreads) {
  double kz = prm[0], cy = prm[1] / (double)(n - 2), cx = prm[2] / ((double)(n - 1) * (double)(n - 2));
  const double* phi = prm + 4;
  /* members of a class as position orders of the triple (i,j,k)/(p,q,r):
   * member 0 = a itself, members 1..5 = the partners b1..b5 of Eq. 2.20 */
  static const int M[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  /* pmap[a][l] = which member is the l-th partner of member a (apply M[l+1] to a's order) */
  int pmap[6][5];
  for (int a = 0; a < 6; a++)
    for (int l = 0; l < 5; l++) {
      int comp[3] = {M[a][M[l + 1][0]], M[a][M[l + 1][1]], M[a][M[l + 1][2]]};
      for (int b = 0; b < 6; b++)
        if (M[b][0] == comp[0] && M[b][1] == comp[1] && M[b][2] == comp[2]) pmap[a][l] = b;
    }
  /* gives[a][b] = weight member a gives to member b */
  double gives[6][6];
  for (int a = 0; a < 6; a++) {
    for (int b = 0; b < 6; b++) gives[a][b] = 0.0;
    for (int l = 0; l < 5; l++) gives[a][pmap[a][l]] = phi[l];
  }
  int uniform = form == 0 && phi[0] == phi[1] && phi[0] == phi[2] && phi[0] == phi[3] && phi[0] == phi[4];
  int folded = variant == 0 && uniform && kz == 1.0;
  double c1 = -(1.0 + phi[0]);
  int ntrip = 0;
  int(*trip)[3] = (int(*)[3])malloc(sizeof(int[3]) * (size_t)(n * n * n / 6 + 1));
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++)
      for (int k = j + 1; k < n; k++) {
        trip[ntrip][0] = i;
        trip[ntrip][1] = j;
        trip[ntrip][2] = k;
        ntrip++;
      }
  /* one canonical class {(i,p),(j,q),(k,r)} with i<j<k at a time: all six s
   * values come from the unmodified snapshot, then the six entries are written */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int tr = 0; tr < ntrip; tr++) {
    int f[3] = {trip[tr][0], trip[tr][1], trip[tr][2]};
    for (int p = 0; p < n; p++)
      for (int q = 0; q < n; q++) {
        if (q == p) continue;
        for (int r = 0; r < n; r++) {
          if (r == p || r == q) continue;
          int l3[3] = {p, q, r};
          double s[6], base[6];
          long long idx[6];
          if (folded) {
            /* kz = 1, all phi equal, S variant: the same pool regrouped,
             * s = (D^ - xi_k') - (psi_r' - ty) and D^' = (D^ + phi S) - (1 + phi) s */
            double Dv[6], S;
            for (int a = 0; a < 6; a++) {
              int fi = f[M[a][0]], fj = f[M[a][1]], fk = f[M[a][2]];
              int li = l3[M[a][0]], lj = l3[M[a][1]], lk = l3[M[a][2]];
              long long t = tile_of(n, fi, li, fj, lj);
              double ty = cy * piy[t] + cx * pix[fi * n + li];
              if (sa) ty = ty + sa[fi * n + li];
              idx[a] = zidx(n, fi, fj, fk, li, lj, lk);
              Dv[a] = Dhat[idx[a]];
              double psi_f = psi[t * (n - 2) + cmp2(lk, li, lj)] - ty;
              s[a] = (Dv[a] - xi[t * (n - 2) + cmp2(fk, fi, fj)]) - psi_f;
            }
            S = s[0];
            for (int b = 1; b < 6; b++) S = S + s[b];
            for (int a = 0; a < 6; a++) Dhat[idx[a]] = fma(c1, s[a], fma(phi[0], S, Dv[a]));
            continue;
          }
          for (int a = 0; a < 6; a++) {
            int fi = f[M[a][0]], fj = f[M[a][1]], fk = f[M[a][2]];
            int li = l3[M[a][0]], lj = l3[M[a][1]], lk = l3[M[a][2]];
            double pz = piz_at(n, Dhat, xi, psi, fi, fj, fk, li, lj, lk);
            double ty = cy * piy[tile_of(n, fi, li, fj, lj)] + cx * pix[fi * n + li];
            if (sa) ty = ty + sa[fi * n + li];
            s[a] = fma(kz, pz, ty);
            idx[a] = zidx(n, fi, fj, fk, li, lj, lk);
            if (variant == 0) {
              base[a] = Dhat[idx[a]] - s[a];
            } else {
              base[a] = fma(-kz, pz, pz);
              if (sa) base[a] = base[a] - sa[fi * n + li];
            }
          }
          double newv[6];
          if (uniform) {
            /* all phi equal: a receives phi * (sum of the other five s) */
            double S = s[0];
            for (int b = 1; b < 6; b++) S = S + s[b];
            for (int a = 0; a < 6; a++) newv[a] = fma(phi[0], S - s[a], base[a]);
          } else {
            /* inflow from a's partners b1..b5 added in that order, one fused
             * multiply-add each, onto the member's own remainder */
            for (int a = 0; a < 6; a++) {
              double acc = base[a];
              for (int l = 0; l < 5; l++) {
                int b = pmap[a][l];
                acc = fma(gives[b][a], s[b], acc);
              }
              newv[a] = acc;
            }
          }
          for (int a = 0; a < 6; a++) Dhat[idx[a]] = newv[a];
        }
      }
  }
  free(trip);
}

void or_redistribute_z_v(int n, const double* prm, int variant, const double* sa, double* Dhat, const double* xi,
                         const double* psi, const double* piy, const double* pix, int nthreads) {
  or_redistribute_z_form(n, prm, variant, sa, 0, Dhat, xi, psi, piy, pix, nthreads);
}

void or_redistribute_z(int n, const double* prm, double* Dhat, const double* xi, const double* psi, const double* piy,
                       const double* pix, int nthreads) {
  or_redistribute_z_v(n, prm, 0, NULL, Dhat, xi, psi, piy, pix, nthreads);
}

/* y redistribution (Type 1 rule for y, Eq. 2.21) in place on C^:
 * C^'_ijpq = (C^_ijpq - phi_y pi_y(ijpq)) + phi_y pi_y(jiqp). */
void or_redistribute_y(int n, double phi_y, double* Chat, const double* piy) {
  long long T = or_num_tiles(n);
  double* out = (double*)malloc(sizeof(double) * T);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      for (int p = 0; p < n; p++)
        for (int q = 0; q < n; q++) {
          if (q == p) continue;
          long long t = tile_of(n, i, p, j, q), tp = tile_of(n, j, q, i, p);
          out[t] = (Chat[t] - phi_y * piy[t]) + phi_y * piy[tp];
        }
    }
  memcpy(Chat, out, sizeof(double) * T);
  free(out);
}

/* F variant (Section 3.4, Psi_2 of Eq. 3.6): the new incremental y cost keeps
 * (1 - ky - phi_y) of its own slack and receives phi_y of its mirror's:
 * C^'_ijpq = keep*pi_y(ijpq) + phi_y*pi_y(jiqp), keep = (1 - ky) - phi_y. */
void or_redistribute_y_fast(int n, double ky, double phi_y, double* Chat, const double* piy) {
  long long T = or_num_tiles(n);
  double keep = (1.0 - ky) - phi_y;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      for (int p = 0; p < n; p++)
        for (int q = 0; q < n; q++) {
          if (q == p) continue;
          long long t = tile_of(n, i, p, j, q), tp = tile_of(n, j, q, i, p);
          Chat[t] = keep * piy[t] + phi_y * piy[tp];
        }
    }
  (void)T;
}

/* F variant: the new incremental x cost is (1 - kx) pi_x (Psi_2 of Eq. 3.6). */
void or_move_x_fast(int n, double kx, double* bx, const double* pix) {
  double keep = 1.0 - kx;
  for (int e = 0; e < n * n; e++) bx[e] = keep * pix[e];
}

/* Second phase of the two-phase Z solve (Section 3.4): for every class
 * (i<j<k, p,q,r distinct) the six members split by their slack into
 * S_B = {pi_z <= tol (1 + |xi_k'| + |psi_r'|)} (zero slack up to the rounding of
 * pi_z = (D^ - xi) - psi) and S_N = the others; every member of S_N drops to
 * D^ - pi_z, and the sum of the S_N slacks (added in member order) times
 * 1/|S_B| is added to every member of S_B.  A class with S_B or S_N empty is
 * left as it is.  All slacks come from one snapshot. */
void or_phase2_z(int n, double tol, double* Dhat, const double* xi, const double* psi, int nthreads) {
  static const int M[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  static const double inv[7] = {0.0, 1.0, 1.0 / 2.0, 1.0 / 3.0, 1.0 / 4.0, 1.0 / 5.0, 1.0 / 6.0};
  int ntrip = n * (n - 1) * (n - 2) / 6;
  int(*trip)[3] = (int(*)[3])malloc(sizeof(int[3]) * (size_t)(ntrip + 1));
  int c = 0;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++)
      for (int k = j + 1; k < n; k++) {
        trip[c][0] = i;
        trip[c][1] = j;
        trip[c][2] = k;
        c++;
      }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int tr = 0; tr < ntrip; tr++) {
    int f[3] = {trip[tr][0], trip[tr][1], trip[tr][2]};
    for (int p = 0; p < n; p++)
      for (int q = 0; q < n; q++) {
        if (q == p) continue;
        for (int r = 0; r < n; r++) {
          if (r == p || r == q) continue;
          int l3[3] = {p, q, r};
          double pz[6];
          long long idx[6];
          int basic[6];
          int nb = 0;
          double sum = 0.0;
          for (int a = 0; a < 6; a++) {
            int fi = f[M[a][0]], fj = f[M[a][1]], fk = f[M[a][2]];
            int li = l3[M[a][0]], lj = l3[M[a][1]], lk = l3[M[a][2]];
            long long t = tile_of(n, fi, li, fj, lj);
            int kk = cmp2(fk, fi, fj), rr = cmp2(lk, li, lj);
            pz[a] = piz_at(n, Dhat, xi, psi, fi, fj, fk, li, lj, lk);
            idx[a] = zidx(n, fi, fj, fk, li, lj, lk);
            double lim = tol * ((1.0 + fabs(xi[t * (n - 2) + kk])) + fabs(psi[t * (n - 2) + rr]));
            basic[a] = pz[a] <= lim;
            if (basic[a]) nb++;
            else sum = sum + pz[a];
          }
          if (nb == 0 || nb == 6) continue;
          double share = sum * inv[nb];
          for (int a = 0; a < 6; a++) {
            if (basic[a]) Dhat[idx[a]] = Dhat[idx[a]] + share;
            else Dhat[idx[a]] = Dhat[idx[a]] - pz[a];
          }
        }
      }
  }
  free(trip);
}

/* Annealing schedule of the Type 4 rule (Section 5): temperature
 * T_0 = t0 * ub, multiplied by `cool` before draws d = period, 2 period, ...;
 * draw d redistributes kappa^lb = sum_i kf[d][i] + sum_p kl[d][p] (facilities
 * first, in index order) of the bound nu when kappa^lb * nu <= e_d * T_d,
 * e_d = -ln(u_d) for the draw's uniform u_d (i.e. u_d <= exp(-kappa^lb nu / T_d)).
 * Outputs K[d] = kappa^lb and thr[d] = e_d * T_d. */
void or_sa_schedule(int n, int count, double ub, double t0, double cool, int period, const double* kf,
                    const double* kl, const double* neglog_u, double* K, double* thr) {
  double T = t0 * ub;
  for (int d = 0; d < count; d++) {
    if (d > 0 && period > 0 && d % period == 0) T = T * cool;
    double k = 0.0;
    for (int i = 0; i < n; i++) k = k + kf[(long long)d * n + i];
    for (int p = 0; p < n; p++) k = k + kl[(long long)d * n + p];
    K[d] = k;
    thr[d] = neglog_u[d] * T;
  }
}

/* Type 4 amounts of one accepted draw (Section 2.3, rule 4): with
 * g = nu / (n (n-1) (n-2)), every z with first facility i and first location p
 * gives up kf[i] g + kl[p] g.  Returns 1 and fills out[n*n] when
 * K * nu <= thr, else returns 0. */
int or_sa_term(int n, double nu, double K, double thr, const double* kf, const double* kl, double* out) {
  if (!(K * nu <= thr)) return 0;
  double c4 = 1.0 / (((double)n * (double)(n - 1)) * (double)(n - 2));
  double g = nu * c4;
  for (int i = 0; i < n; i++)
    for (int p = 0; p < n; p++) out[i * n + p] = kf[i] * g + kl[p] * g;
  return 1;
}

/* Feasibility check (Section 2.3, after Algorithm 1): build y and z from the
 * X-LAP primal and test complementary slackness (Eq. 2.19) for them. */
int or_feasibility(int n, const int* xperm, const double* piy, const double* Dhat, const double* xi, const double* psi,
                   double tol) {
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      if (fabs(piy[tile_of(n, i, xperm[i], j, xperm[j])]) > tol) return 0;
      for (int k = 0; k < n; k++) {
        if (k == i || k == j) continue;
        if (fabs(piz_at(n, Dhat, xi, psi, i, j, k, xperm[i], xperm[j], xperm[k])) > tol) return 0;
      }
    }
  return 1;
}

/* One S1 iteration (Algorithm 1 steps 3-5, then the ascent step).  u0z, u0y,
 * u0x (nullable): starting row duals of the Z, Y and X LAPs (warm starts).
 * prm = {kz, ky, kx, phi_y, phi_1..phi_5}; stats[6] = {aug,relax} for Z, Y, X. */
int or_iterate(int n, const double* prm, int dual_mode, const double* bprime, double* Chat, double* Dhat,
               const double* u0z, const double* u0y, const double* u0x, double* lb, double* Theta, double* xi, double* psi, double* Delta, double* gamma,
               double* delta, double* alpha, double* beta, int* xperm, double* pix, double* piy, long long* stats,
               int nthreads) {
  if (n < 3) return OR_EINVAL;
  long long st[6] = {0, 0, 0, 0, 0, 0};
  or_stage_z(n, dual_mode, Dhat, u0z, Theta, xi, psi, &st[0], &st[1], nthreads);
  or_stage_y(n, dual_mode, Chat, Theta, u0y, Delta, gamma, delta, &st[2], &st[3]);
  or_stage_x(n, dual_mode, bprime, Delta, u0x, lb, alpha, beta, xperm, &st[4], &st[5]);
  or_reduced_xy(n, bprime, Delta, alpha, beta, Chat, Theta, gamma, delta, pix, piy);
  or_redistribute_z(n, prm, Dhat, xi, psi, piy, pix, nthreads);
  or_redistribute_y(n, prm[3], Chat, piy);
  if (stats) memcpy(stats, st, sizeof st);
  return OR_OK;
}

/* One iteration of any variant of Section 3.4 (S or F; one or two phases;
 * with or without the Type 4 rule), then its ascent step.
 * opt = {dual_mode, variant (0 S, 1 F), two_phase, warm2}: warm2 = 1 starts the
 * second Z solve from the first solve's row duals; p2tol is the second phase's
 * zero-slack tolerance.
 * lb_base: S passes the constant of the fixed facilities; F passes the
 * previous bound (the constant before the first iteration); *lb = lb_base + the
 * X-LAP value (for F the previous bound plus the increment, Eq. 3.7).
 * bx: x costs (b' in S; the incremental x cost in F, updated in place).
 * sa_draw (nullable): {K, thr} of this iteration's draw with kf, kl (n each);
 * *sa_on reports whether the draw was accepted at the new bound. */
int or_iterate_v(int n, const double* prm, const int* opt, double p2tol, double lb_base, double* bx, double* Chat, double* Dhat,
                 const double* u0z, const double* u0y, const double* u0x, const double* sa_draw, const double* kf,
                 const double* kl, double* lb, double* Theta, double* xi, double* psi, double* Delta, double* gamma,
                 double* delta, double* alpha, double* beta, int* xperm, double* pix, double* piy, int* sa_on,
                 long long* stats, int nthreads) {
  if (n < 3) return OR_EINVAL;
  int dual_mode = opt[0], variant = opt[1], two_phase = opt[2], warm2 = opt[3];
  long long st[6] = {0, 0, 0, 0, 0, 0};
  long long T = or_num_tiles(n);
  int m = n - 2;
  or_stage_z(n, dual_mode, Dhat, u0z, Theta, xi, psi, &st[0], &st[1], nthreads);
  if (two_phase) {
    long long a2 = 0, r2 = 0;
    double* u1 = NULL;
    or_phase2_z(n, p2tol, Dhat, xi, psi, nthreads);
    if (warm2) {
      u1 = (double*)malloc(sizeof(double) * (size_t)(T * m));
      memcpy(u1, xi, sizeof(double) * (size_t)(T * m));
    }
    or_stage_z(n, dual_mode, Dhat, u1, Theta, xi, psi, &a2, &r2, nthreads);
    free(u1);
    st[0] += a2;
    st[1] += r2;
  }
  double xv = 0.0;
  or_stage_y(n, dual_mode, Chat, Theta, u0y, Delta, gamma, delta, &st[2], &st[3]);
  or_stage_x(n, dual_mode, bx, Delta, u0x, &xv, alpha, beta, xperm, &st[4], &st[5]);
  *lb = lb_base + xv;
  or_reduced_xy(n, bx, Delta, alpha, beta, Chat, Theta, gamma, delta, pix, piy);
  double* sa = NULL;
  *sa_on = 0;
  if (sa_draw) {
    sa = (double*)malloc(sizeof(double) * n * n);
    *sa_on = or_sa_term(n, *lb, sa_draw[0], sa_draw[1], kf, kl, sa);
    if (!*sa_on) {
      free(sa);
      sa = NULL;
    }
  }
  or_redistribute_z_v(n, prm, variant, sa, Dhat, xi, psi, piy, pix, nthreads);
  if (variant == 0) {
    or_redistribute_y(n, prm[3], Chat, piy);
  } else {
    or_redistribute_y_fast(n, prm[1], prm[3], Chat, piy);
    or_move_x_fast(n, prm[2], bx, pix);
  }
  free(sa);
  if (stats) memcpy(stats, st, sizeof st);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Half-Z-LAP scheme (Section 5, after Goncalves et al.).  Members of a class  */
/* whose first facility index exceeds the second ("lower order") keep cost 0:  */
/* their Z-LAPs (i > j) have optimum 0 and zero duals and are not solved.     */
/* The three upper members (i,j,k|p,q,r), (i,k,j|p,r,q), (j,k,i|q,r,p) pool   */
/* s = kz pi_z + cy pi'_y + cx pi_x, pi'_y the upper y's slack after the y    */
/* move of Eq. 2.21 (phi_y = 1/2), and each takes half of the other two      */
/* pools; a lower y passes kx pi_x/(n-1) to its mirror on the y level.        */
/* ------------------------------------------------------------------------ */
void or_stage_z_upper(int n, int dual_mode, const double* Dhat, const double* u0, double* Theta, double* xi,
                      double* psi, long long* naug, long long* nrelax) {
  int m = n - 2;
  long long aug_tot = 0, relax_tot = 0;
  for (int i = 0; i < n; i++)
    for (int p = 0; p < n; p++)
      for (int j = 0; j < n; j++) {
        if (j == i) continue;
        for (int q = 0; q < n; q++) {
          if (q == p) continue;
          long long t = tile_of(n, i, p, j, q);
          if (j < i) {
            Theta[t] = 0.0;
            for (int k = 0; k < m; k++) xi[t * m + k] = psi[t * m + k] = 0.0;
            continue;
          }
          int perm[64];
          int aug;
          long long relax;
          solve_one(m, Dhat + t * m * m, u0 ? u0 + t * m : NULL, dual_mode, &Theta[t], xi + t * m, psi + t * m, perm,
                    &aug, &relax);
          aug_tot += aug;
          relax_tot += relax;
        }
      }
  if (naug) *naug = aug_tot;
  if (nrelax) *nrelax = relax_tot;
}

/* form 0: the regrouped member update (D + S/2) - (3/2) s; form 1: the plain
 * definition (D - s) + s_b/2 + s_c/2, the two other upper members' pools added
 * one at a time in member order (the reference the regrouping is tested against). */
void or_redistribute_half_form(int n, const double* prm, int form, double* Dhat, double* Chat, const double* xi,
                               const double* psi, const double* piy, const double* pix) {
  double kz = prm[0], cy = prm[1] / (double)(n - 2), cx = prm[2] / ((double)(n - 1) * (double)(n - 2));
  double phi_y = prm[3], cxy = prm[2] / (double)(n - 1);
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++)
      for (int k = j + 1; k < n; k++)
        for (int p = 0; p < n; p++)
          for (int q = 0; q < n; q++) {
            if (q == p) continue;
            for (int r = 0; r < n; r++) {
              if (r == p || r == q) continue;
              /* upper members in member order: (i,j,k|p,q,r), (i,k,j|p,r,q), (j,k,i|q,r,p) */
              int F[3][3] = {{i, j, k}, {i, k, j}, {j, k, i}};
              int L[3][3] = {{p, q, r}, {p, r, q}, {q, r, p}};
              double s[3], D[3];
              long long idx[3];
              for (int u = 0; u < 3; u++) {
                int a = F[u][0], b = F[u][1], c = F[u][2], x = L[u][0], y = L[u][1], w = L[u][2];
                double pz = piz_at(n, Dhat, xi, psi, a, b, c, x, y, w);
                /* the upper y's slack after the y move: its own half kept plus half of its mirror's */
                long long t = tile_of(n, a, x, b, y), tm = tile_of(n, b, y, a, x);
                double py = (piy[t] - phi_y * piy[t]) + phi_y * piy[tm];
                double ty = cy * py + cx * pix[a * n + x];
                s[u] = fma(kz, pz, ty);
                idx[u] = zidx(n, a, b, c, x, y, w);
                D[u] = Dhat[idx[u]];
              }
              if (form == 1) {
                for (int u = 0; u < 3; u++) {
                  double acc = D[u] - s[u];
                  for (int w = 0; w < 3; w++)
                    if (w != u) acc = acc + 0.5 * s[w];
                  Dhat[idx[u]] = acc;
                }
                continue;
              }
              double S = (s[0] + s[1]) + s[2];
              /* D - s + (S - s)/2, regrouped as (D + S/2) - (3/2) s */
              for (int u = 0; u < 3; u++) Dhat[idx[u]] = fma(-1.5, s[u], fma(0.5, S, D[u]));
            }
          }
  /* y move of Eq. 2.21 with phi_y (1/2): every y keeps (1 - phi_y) of its slack and
   * receives phi_y of its mirror's; an upper y then gives that updated slack to its z (ky) */
  long long T = or_num_tiles(n);
  double* out = (double*)malloc(sizeof(double) * T);
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      for (int p = 0; p < n; p++)
        for (int q = 0; q < n; q++) {
          if (q == p) continue;
          long long t = tile_of(n, i, p, j, q), tp = tile_of(n, j, q, i, p);
          out[t] = (Chat[t] - phi_y * piy[t]) + phi_y * piy[tp];
          /* Type 3 on the y level for the lower rows: y_ijpq (i > j) gives
           * kx pi_x(ip) / (n-1) to its mirror y_jiqp */
          if (i > j) out[t] = out[t] - cxy * pix[i * n + p];
          else out[t] = out[t] + cxy * pix[j * n + q];
        }
    }
  memcpy(Chat, out, sizeof(double) * T);
  free(out);
}

void or_redistribute_half(int n, const double* prm, double* Dhat, double* Chat, const double* xi, const double* psi,
                          const double* piy, const double* pix) {
  or_redistribute_half_form(n, prm, 0, Dhat, Chat, xi, psi, piy, pix);
}

/* One iteration of the half-Z scheme (solve, then the ascent step in place).
 * prm = {kz, ky, kx, phi_y} (the paper: 2/3, 1, 1, 1/2). */
int or_iterate_half(int n, const double* prm, int dual_mode, const double* bprime, double* Chat, double* Dhat,
                    const double* u0z, const double* u0y, const double* u0x, double* lb, double* Theta, double* xi,
                    double* psi, double* Delta, double* gamma, double* delta, double* alpha, double* beta,
                    int* xperm, double* pix, double* piy, long long* stats) {
  if (n < 3) return OR_EINVAL;
  long long st[6] = {0, 0, 0, 0, 0, 0};
  or_stage_z_upper(n, dual_mode, Dhat, u0z, Theta, xi, psi, &st[0], &st[1]);
  or_stage_y(n, dual_mode, Chat, Theta, u0y, Delta, gamma, delta, &st[2], &st[3]);
  or_stage_x(n, dual_mode, bprime, Delta, u0x, lb, alpha, beta, xperm, &st[4], &st[5]);
  or_reduced_xy(n, bprime, Delta, alpha, beta, Chat, Theta, gamma, delta, pix, piy);
  or_redistribute_half(n, prm, Dhat, Chat, xi, psi, piy, pix);
  if (stats) memcpy(stats, st, sizeof st);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Parent -> child warm start of the branch-and-bound (Section 4, step 3):   */
/* fixing facility f at location l (residual indices of the parent) in the  */
/* parent's Lagrangian LRLT2(v) turns y_{i f p l}, y_{f i l p} into x_ip and  */
/* z with (f,l) in any position into the y of the other two, so the child's */
/* multiplier-adjusted costs are                                             */
/*   D^_c(i,j,k|p,q,r) = D^_p(same facilities and locations)                 */
/*   C^_c(i,j|p,q) = ((C^_p(i,j|p,q) + D^_p(i,j,f|p,q,l)) + D^_p(i,f,j|p,l,q)) */
/*                   + D^_p(f,i,j|l,p,q)                                     */
/*   b'_c(i|p)     = (b'_p(i|p) + C^_p(i,f|p,l)) + C^_p(f,i|l,p)              */
/*   const_c       = const_p + b'_p(f|l)                                     */
/* (child residual index a <-> parent a + (a >= f), locations likewise).      */
/* ------------------------------------------------------------------------ */
void or_child_state(int np, int f, int l, const double* bp, const double* Cp, const double* Dp, double cst_p,
                    double* bc, double* Cc, double* Dc, double* cst_c) {
  int nc = np - 1;
#define PF(a) ((a) + ((a) >= f))
#define PL(a) ((a) + ((a) >= l))
  *cst_c = cst_p + bp[f * np + l];
  for (int i = 0; i < nc; i++)
    for (int p = 0; p < nc; p++) {
      int I = PF(i), P = PL(p);
      bc[i * nc + p] = (bp[I * np + P] + Cp[tile_of(np, I, P, f, l)]) + Cp[tile_of(np, f, l, I, P)];
    }
  for (int i = 0; i < nc; i++)
    for (int j = 0; j < nc; j++) {
      if (j == i) continue;
      for (int p = 0; p < nc; p++)
        for (int q = 0; q < nc; q++) {
          if (q == p) continue;
          int I = PF(i), J = PF(j), P = PL(p), Q = PL(q);
          double c = Cp[tile_of(np, I, P, J, Q)];
          if (nc >= 2 && np >= 3) {
            c = c + Dp[zidx(np, I, J, f, P, Q, l)];
            c = c + Dp[zidx(np, I, f, J, P, l, Q)];
            c = c + Dp[zidx(np, f, I, J, l, P, Q)];
          }
          Cc[tile_of(nc, i, p, j, q)] = c;
          if (nc < 3) continue;
          for (int k = 0; k < nc; k++) {
            if (k == i || k == j) continue;
            for (int r = 0; r < nc; r++) {
              if (r == p || r == q) continue;
              Dc[zidx(nc, i, j, k, p, q, r)] = Dp[zidx(np, I, J, PF(k), P, Q, PL(r))];
            }
          }
        }
    }
#undef PF
#undef PL
}

/* Lagrangian objective of one full assignment (perm over the residual
 * problem): const + sum_i b'(i|s_i) + sum_{i!=j} C^(i,j|s_i,s_j)
 * + sum_{i,j,k distinct} D^(i,j,k|s_i,s_j,s_k).  For a permutation every RLT2
 * constraint holds, so this equals the QAP cost for any multipliers. */
double or_lagrangian_objective(int n, const double* b, const double* C, const double* D, double cst, const int* s) {
  double v = cst;
  for (int i = 0; i < n; i++) v += b[i * n + s[i]];
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) {
      if (j == i) continue;
      v += C[tile_of(n, i, s[i], j, s[j])];
      if (n < 3) continue;
      for (int k = 0; k < n; k++) {
        if (k == i || k == j) continue;
        v += D[zidx(n, i, j, k, s[i], s[j], s[k])];
      }
    }
  return v;
}

int or_have_openmp(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 0;
#endif
}

/* ------------------------------------------------------------------------ */
/* Learned warm start (not in the paper): features, FP64 reference MLP.     */
/* ------------------------------------------------------------------------ */
/* FP64 -> FP32 by truncating the significand (exponent clamped to the FP32
 * range; below it -> signed zero, above it -> +-FLT_MAX).  Done on bits so the
 * GPU can reproduce it with integer instructions. */
float or_f32_trunc(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  uint32_t sign = (uint32_t)(b >> 63) << 31;
  int e = (int)((b >> 52) & 0x7ff);
  uint32_t out;
  if (e == 0) {
    out = sign;
  } else {
    int ef = e - 1023 + 127;
    if (ef <= 0) out = sign;
    else if (ef >= 255) out = sign | 0x7f7fffffu;
    else out = sign | ((uint32_t)ef << 23) | (uint32_t)((b >> 29) & 0x7fffff);
  }
  float f;
  memcpy(&f, &out, 4);
  return f;
}

/* FP32 -> BF16 (round to nearest even), returned as the FP32 value it represents. */
float or_bf16_round(float x) {
  uint32_t b;
  memcpy(&b, &x, 4);
  uint32_t lsb = (b >> 16) & 1u;
  b = (b + 0x7fffu + lsb) & 0xffff0000u;
  float f;
  memcpy(&f, &b, 4);
  return f;
}

#define OR_MLP_IN 34
/* Row features of one m x m tile (m <= 32), all in FP32:
 *  cf = trunc32(c); colmin_j = min_i cf_ij; R = cf - colmin;
 *  s = max R (1 if 0); inv = 1/s; row i: sort(R_i * inv) ascending, padded with
 *  zeros to 32; feature 32 = trunc32(prev_u_i) * inv (0 without prev);
 *  feature 33 = m/32.  Target (optional): the change of the row dual,
 *  trunc32(u*_i - prev_u_i) * inv (trunc32(u*_i) * inv without prev). */
void or_mlp_features(int m, const double* tile, const double* prev_u, const double* target_u, float* feat,
                     float* target_out, float* scale_out) {
  float cf[32 * 32], cmin[32], s = 0.0f;
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) cf[i * 32 + j] = or_f32_trunc(tile[i * m + j]);
  for (int j = 0; j < m; j++) {
    float mn = cf[j];
    for (int i = 1; i < m; i++)
      if (cf[i * 32 + j] < mn) mn = cf[i * 32 + j];
    cmin[j] = mn;
  }
  for (int i = 0; i < m; i++)
    for (int j = 0; j < m; j++) {
      float r = cf[i * 32 + j] - cmin[j];
      if (r > s) s = r;
    }
  if (!(s > 0.0f)) s = 1.0f;
  float inv = 1.0f / s;
  for (int i = 0; i < m; i++) {
    float row[32];
    for (int j = 0; j < m; j++) row[j] = (cf[i * 32 + j] - cmin[j]) * inv;
    for (int a = 1; a < m; a++) { /* insertion sort */
      float x = row[a];
      int b = a - 1;
      while (b >= 0 && row[b] > x) {
        row[b + 1] = row[b];
        b--;
      }
      row[b + 1] = x;
    }
    for (int k = 0; k < 32; k++) feat[i * OR_MLP_IN + k] = k < m ? row[k] : 0.0f;
    feat[i * OR_MLP_IN + 32] = prev_u ? or_f32_trunc(prev_u[i]) * inv : 0.0f;
    feat[i * OR_MLP_IN + 33] = (float)m / 32.0f;
    if (target_u && target_out) target_out[i] = or_f32_trunc(prev_u ? target_u[i] - prev_u[i] : target_u[i]) * inv;
  }
  if (scale_out) *scale_out = s;
}

/* FP64 forward pass of the 3-layer MLP on N rows of 34 features:
 *  h1 = relu(X W1 + b1), h2 = relu(h1 W2 + b2), out = h2 . w3 + b3,
 *  W1: 34 x H, W2: H x H (row-major, input index first).  With bf16_acts the
 *  inputs of every matrix product (X, h1, h2) are rounded to BF16, as the
 *  tensor-core path stores them. */
void or_mlp_forward(int N, int H, const float* X, const float* W1, const float* b1, const float* W2,
                    const float* b2, const float* w3, double b3, int bf16_acts, double* out, double* h1,
                    double* h2) {
  for (int r = 0; r < N; r++) {
    double* a1 = h1 + (size_t)r * H;
    double* a2 = h2 + (size_t)r * H;
    for (int j = 0; j < H; j++) {
      double s = b1[j];
      for (int k = 0; k < OR_MLP_IN; k++) {
        double x = bf16_acts ? (double)or_bf16_round(X[r * OR_MLP_IN + k]) : (double)X[r * OR_MLP_IN + k];
        s += x * (double)W1[k * H + j];
      }
      a1[j] = s > 0.0 ? s : 0.0;
      if (bf16_acts) a1[j] = (double)or_bf16_round((float)a1[j]);
    }
    for (int j = 0; j < H; j++) {
      double s = b2[j];
      for (int k = 0; k < H; k++) s += a1[k] * (double)W2[(size_t)k * H + j];
      a2[j] = s > 0.0 ? s : 0.0;
      if (bf16_acts) a2[j] = (double)or_bf16_round((float)a2[j]);
    }
    double s = b3;
    for (int k = 0; k < H; k++) s += a2[k] * (double)w3[k];
    out[r] = s;
  }
}

/* Gradients of L = 1/(2N) sum_r (out_r - t_r)^2 (after or_mlp_forward with the
 * same arguments).  With bf16_acts the back-propagated activation gradients
 * dh2 and dh1 are rounded to BF16 where the tensor-core path stores them. */
double or_mlp_backward(int N, int H, const float* X, const float* W2, const float* w3, int bf16_acts,
                       const double* out, const double* h1, const double* h2, const double* t, double* gW1,
                       double* gb1, double* gW2, double* gb2, double* gw3, double* gb3) {
  double loss = 0.0;
  memset(gW1, 0, sizeof(double) * OR_MLP_IN * H);
  memset(gb1, 0, sizeof(double) * H);
  memset(gW2, 0, sizeof(double) * (size_t)H * H);
  memset(gb2, 0, sizeof(double) * H);
  memset(gw3, 0, sizeof(double) * H);
  *gb3 = 0.0;
  double* d2 = (double*)malloc(sizeof(double) * H);
  double* d1 = (double*)malloc(sizeof(double) * H);
  for (int r = 0; r < N; r++) {
    double e = out[r] - t[r];
    loss += 0.5 * e * e / N;
    double dout = e / N;
    const double* a1 = h1 + (size_t)r * H;
    const double* a2 = h2 + (size_t)r * H;
    *gb3 += dout;
    for (int k = 0; k < H; k++) {
      gw3[k] += a2[k] * dout;
      d2[k] = a2[k] > 0.0 ? dout * (double)w3[k] : 0.0;
      if (bf16_acts) d2[k] = (double)or_bf16_round((float)d2[k]);
    }
    for (int j = 0; j < H; j++) {
      gb2[j] += d2[j];
      for (int k = 0; k < H; k++) gW2[(size_t)k * H + j] += a1[k] * d2[j];
    }
    for (int k = 0; k < H; k++) {
      double s = 0.0;
      for (int j = 0; j < H; j++) s += (double)W2[(size_t)k * H + j] * d2[j];
      d1[k] = a1[k] > 0.0 ? s : 0.0;
      if (bf16_acts) d1[k] = (double)or_bf16_round((float)d1[k]);
    }
    for (int j = 0; j < H; j++) {
      gb1[j] += d1[j];
      for (int k = 0; k < OR_MLP_IN; k++) {
        double x = bf16_acts ? (double)or_bf16_round(X[r * OR_MLP_IN + k]) : (double)X[r * OR_MLP_IN + k];
        gW1[k * H + j] += x * d1[j];
      }
    }
  }
  free(d2);
  free(d1);
  return loss;
}
