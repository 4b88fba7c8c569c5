"""The oracle's C code under AddressSanitizer and UndefinedBehaviorSanitizer.

A small C driver (written here) links the oracle sources built with
-fsanitize=address,undefined (every report fatal) and OpenMP, and calls every
entry point of oracle/oracle.h on a Kuhn box of 3 x 3 x 3 cubes (162 tets)
with an affine-plus-quadratic magnetisation: the single-tet integrals (closed
form, cone quadrature, 3-D Gauss), the direct sum, the charge routes for u and
for the pointwise field, lumped H, moments and translations, and the tree and
FMM for the three source models, on two threads.  Any out-of-bounds access,
use after free, leak, signed overflow, misaligned or invalid value stops it
with a non-zero status."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

DRIVER = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define N 3
static int nid(int i, int j, int k) { return (i * (N + 1) + j) * (N + 1) + k; }

int main(void) {
  const int nn = (N + 1) * (N + 1) * (N + 1), nt = 6 * N * N * N, B = 2;
  double* nodes = malloc(sizeof(double) * 3 * nn);
  int32_t* tets = malloc(sizeof(int32_t) * 4 * nt);
  for (int i = 0; i <= N; i++)
    for (int j = 0; j <= N; j++)
      for (int k = 0; k <= N; k++) {
        double* x = nodes + 3 * nid(i, j, k);
        x[0] = i; x[1] = j; x[2] = k;
      }
  /* each cube: the six paths v -> v+e_a -> v+e_a+e_b -> v+(1,1,1) */
  static const int perm[6][3] = {{0,1,2},{0,2,1},{1,0,2},{1,2,0},{2,0,1},{2,1,0}};
  int t = 0;
  for (int i = 0; i < N; i++)
    for (int j = 0; j < N; j++)
      for (int k = 0; k < N; k++)
        for (int q = 0; q < 6; q++) {
          int c[3] = {i, j, k};
          tets[4 * t] = nid(c[0], c[1], c[2]);
          for (int s = 0; s < 3; s++) {
            c[perm[q][s]]++;
            tets[4 * t + 1 + s] = nid(c[0], c[1], c[2]);
          }
          t++;
        }
  double* M = malloc(sizeof(double) * B * nn * 3);
  for (int b = 0; b < B; b++)
    for (int i = 0; i < nn; i++) {
      const double* x = nodes + 3 * i;
      M[(b * nn + i) * 3 + 0] = 1.0 + 0.1 * x[1] + 0.02 * b * x[2] * x[2];
      M[(b * nn + i) * 3 + 1] = 0.3 - 0.2 * x[0] * x[2];
      M[(b * nn + i) * 3 + 2] = 0.5 + 0.05 * x[0] + b;
    }
  double sum = 0.0;

  /* single tet */
  const double v[12] = {0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 1};
  const double Mt[12] = {1, 0, 0, 0.5, 0.2, 0, 0, 1, 0.3, 0.1, 0.1, 1};
  const double r[3] = {0.3, 0.2, 0.1}, rf[3] = {3.0, -2.0, 1.5};
  sum += oracle_tet_potential(r, v, Mt) + oracle_tet_potential_cone_quad(r, v, Mt, 1e-8) +
         oracle_tet_potential_gauss3d(rf, v, Mt, 6);

  /* whole mesh, direct sum and lumped H */
  double* u = calloc((size_t)B * nn, sizeof(double));
  double* H = calloc((size_t)B * nn * 3, sizeof(double));
  double* vol = malloc(sizeof(double) * nt);
  if (oracle_direct(nodes, nn, tets, nt, M, B, NULL, nn, u, 2)) return 10;
  if (oracle_lumped_H(nodes, nn, tets, nt, u, B, H)) return 11;
  oracle_tet_volumes(nodes, tets, nt, vol);
  for (int i = 0; i < B * nn; i++) sum += u[i] + H[3 * i];

  /* charge routes: boundary faces (face f opposite vertex f) on the box planes */
  int32_t* bf = malloc(sizeof(int32_t) * 2 * 4 * nt);
  int nbf = 0;
  for (int e = 0; e < nt; e++)
    for (int f = 0; f < 4; f++)
      for (int a = 0; a < 3; a++)
        for (int side = 0; side <= N; side += N) {
          int on = 1;
          for (int q = 0; q < 4; q++)
            if (q != f && nodes[3 * tets[4 * e + q] + a] != side) on = 0;
          if (on) { bf[2 * nbf] = e; bf[2 * nbf + 1] = f; nbf++; }
        }
  if (nbf != 2 * 6 * N * N) return 12;
  int64_t tg[3] = {0, nid(1, 1, 1), nn - 1};
  double uc[2 * 3];
  if (oracle_direct_charges(nodes, nn, tets, nt, bf, nbf, M, B, tg, 3, uc, 2)) return 13;
  const double pts[6] = {1.37, 1.61, 1.23, 0.7, 2.2, 1.3};  /* on no face or edge of the Kuhn tets */
  double Hp[2 * 2 * 3];
  if (oracle_field_charges(nodes, nn, tets, nt, bf, nbf, M, B, pts, 2, Hp, 2)) return 14;
  for (int i = 0; i < 6; i++) sum += uc[i];
  for (int i = 0; i < 12; i++) sum += Hp[i];

  /* expansions */
  const int p = 6, nc = oracle_ncoef(p);
  int32_t* mi = malloc(sizeof(int32_t) * 3 * nc);
  double *D = malloc(sizeof(double) * oracle_ncoef(2 * p)), *Q = calloc(nc, sizeof(double)),
         *Qp = calloc(nc, sizeof(double)), *L = calloc(nc, sizeof(double)), *Lc = calloc(nc, sizeof(double));
  oracle_multi_indices(p, mi);
  const double x[3] = {2.0, -1.0, 0.5}, c[3] = {0.25, 0.25, 0.25}, d[3] = {0.1, -0.2, 0.05};
  oracle_laplace_derivs(x, 2 * p, D);
  oracle_tet_moments(v, Mt, c, p, Q);
  sum += oracle_tet_lambda_monomial_exact(v, c, 2, 1, 2, 0);
  oracle_m2m(p, d, Q, Qp);
  oracle_m2l(p, x, Qp, L);
  oracle_l2l(p, d, L, Lc);
  sum += oracle_l2p(p, d, Lc) + oracle_multipole_eval(p, c, Q, rf) + D[nc - 1];

  /* tree and FMM, three source models */
  for (int src = 0; src < 3; src++) {
    int st = 0;
    oracle_tree* tr = oracle_tree_build_sources(nodes, nn, tets, nt, 8, 0.5, src, &st);
    if (!tr || st) return 20 + src;
    int64_t info[5];
    double box[5];
    oracle_tree_info(tr, info);
    oracle_tree_box(tr, box);
    const int64_t ncl = info[0], nm = info[1], np = info[2];
    uint64_t *nk = malloc(8 * nn), *tk = malloc(8 * nt), *pre = malloc(8 * ncl);
    int64_t *npm = malloc(8 * nn), *tpm = malloc(8 * nt), *rng = malloc(8 * 4 * ncl), *par = malloc(8 * ncl),
            *chi = malloc(8 * 2 * ncl), *mo = malloc(8 * (ncl + 1)), *ms = malloc(8 * (nm + 1)),
            *po = malloc(8 * (ncl + 1)), *ps = malloc(8 * (np + 1));
    int32_t* lev = malloc(4 * ncl);
    double *cen = malloc(8 * 3 * ncl), *rad = malloc(8 * 2 * ncl);
    oracle_tree_export(tr, nk, tk, npm, tpm, lev, pre, rng, par, chi, cen, rad, mo, ms, po, ps);
    double* uf = calloc((size_t)B * nn, sizeof(double));
    if (oracle_fmm_eval(tr, 4, M, B, uf, NULL, 0, 2)) return 30 + src;
    int64_t leaves[2], nl = 0;
    for (int64_t q = 0; q < ncl && nl < 2; q++)
      if (chi[2 * q + 1] == 0 && rng[4 * q + 3] > rng[4 * q + 2]) leaves[nl++] = q;
    if (oracle_fmm_eval(tr, 4, M, B, uf, leaves, nl, 1)) return 40 + src;
    for (int i = 0; i < B * nn; i++) sum += uf[i];
    free(nk); free(tk); free(pre); free(npm); free(tpm); free(rng); free(par); free(chi);
    free(mo); free(ms); free(po); free(ps); free(lev); free(cen); free(rad); free(uf);
    oracle_tree_free(tr);
  }
  free(nodes); free(tets); free(M); free(u); free(H); free(vol); free(bf); free(mi); free(D); free(Q); free(Qp);
  free(L); free(Lc);
  if (!isfinite(sum)) return 50;
  printf("ok %.6e\n", sum);
  return 0;
}
"""

FLAGS = ["-O1", "-g", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-omit-frame-pointer",
         "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]


def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    drv = tmp_path / "driver.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "oracle_sanitized"
    srcs = [os.path.join(ORACLE, s) for s in ("oracle_direct.c", "oracle_fmm.c")]
    r = subprocess.run([gcc, *FLAGS, "-I", ORACLE, str(drv), *srcs, "-lm", "-o", str(exe)], capture_output=True,
                       text=True)
    if r.returncode and "asan" in (r.stderr or "").lower():
        pytest.skip("sanitizer runtime not available: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1",
               OMP_NUM_THREADS="2")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.returncode, r.stdout[-500:], r.stderr[-4000:])
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-4000:]
