"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host only): a driver builds graphs in C
(grids with ties, a random graph with a random spanning tree, a path, a forest) and runs every oracle entry point
-- both scoring methods, the recovery at several budgets and c, both spanning trees -- with the sanitizers on."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int orc_offtree_scores(int64_t, const int64_t*, const int32_t*, const double*, const int32_t*, int32_t, int, int,
                       int64_t*, int32_t*, int32_t*, int32_t*, int32_t*, double*, double*, int32_t*);
int orc_recover(int64_t, const int64_t*, const int32_t*, const double*, const int32_t*, double, int32_t, int, int64_t,
                int32_t*, double*, int64_t, int64_t*, int64_t*);
int orc_spanning_tree(int64_t, const int64_t*, const int32_t*, const double*, int, int32_t*);
double orc_exact_sum(const double*, int64_t);

/* symmetric CSR of an undirected edge list (neighbours sorted) */
static void csr(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const double* ew, int64_t* rp,
                int32_t* col, double* w) {
  for (int64_t v = 0; v <= n; v++) rp[v] = 0;
  for (int64_t e = 0; e < m; e++) { rp[eu[e] + 1]++; rp[ev[e] + 1]++; }
  for (int64_t v = 0; v < n; v++) rp[v + 1] += rp[v];
  int64_t* fill = calloc((size_t)n, sizeof(int64_t));
  for (int64_t e = 0; e < m; e++) {
    col[rp[eu[e]] + fill[eu[e]]] = ev[e]; w[rp[eu[e]] + fill[eu[e]]++] = ew[e];
    col[rp[ev[e]] + fill[ev[e]]] = eu[e]; w[rp[ev[e]] + fill[ev[e]]++] = ew[e];
  }
  for (int64_t v = 0; v < n; v++)  /* insertion sort of each row */
    for (int64_t p = rp[v] + 1; p < rp[v + 1]; p++) {
      int32_t c = col[p]; double x = w[p]; int64_t q = p - 1;
      while (q >= rp[v] && col[q] > c) { col[q + 1] = col[q]; w[q + 1] = w[q]; q--; }
      col[q + 1] = c; w[q + 1] = x;
    }
  free(fill);
}

/* forest: the recovery entry points must reject the two roots (error paths run under the sanitizers too) */
static int run(const char* name, int64_t n, int64_t m, const int32_t* eu, const int32_t* ev, const double* ew,
               int forest) {
  int64_t* rp = malloc(sizeof(int64_t) * (n + 1));
  int32_t* col = malloc(sizeof(int32_t) * (2 * m + 1));
  double* w = malloc(sizeof(double) * (2 * m + 1));
  int32_t* parent = malloc(sizeof(int32_t) * n);
  int64_t E = m - n + 2;
  int32_t *u = malloc(sizeof(int32_t) * E), *v = malloc(sizeof(int32_t) * E), *id = malloc(sizeof(int32_t) * E);
  int32_t *l = malloc(sizeof(int32_t) * E), *b = malloc(sizeof(int32_t) * E);
  double *r = malloc(sizeof(double) * E), *s = malloc(sizeof(double) * E);
  int32_t* ids = malloc(sizeof(int32_t) * (m + 1));
  double* sc = malloc(sizeof(double) * (m + 1));
  csr(n, m, eu, ev, ew, rp, col, w);
  int bad = 0;
  for (int kind = 0; kind < 2; kind++) {
    int st = orc_spanning_tree(n, rp, col, w, kind, parent);
    if (st != 0) { if (kind == 0) bad |= 1; continue; }  /* kind 1 needs a connected graph */
    for (int method = 0; method < 2; method++) {
      int64_t noff = 0;
      if ((orc_offtree_scores(n, rp, col, w, parent, 2, 0, method, &noff, u, v, id, l, r, s, b) != 0) != forest)
        bad |= 2;
    }
    for (int c = 0; c <= 3; c++)
      for (int a = 0; a < 3; a++) {
        int64_t cnt = 0, full = 0;
        const double alpha[3] = {0.02, 0.1, 0.5};
        if ((orc_recover(n, rp, col, w, parent, alpha[a], c, a & 1, -1, ids, sc, m + 1, &cnt, &full) < 0) != forest)
          bad |= 4;
      }
  }
  double xs[3] = {1e-300, 1.0, 1e300};
  if (orc_exact_sum(xs, 3) != 1e300) bad |= 8;
  printf("%s: %s\n", name, bad ? "FAIL" : "ok");
  free(rp); free(col); free(w); free(parent); free(u); free(v); free(id); free(l); free(b); free(r); free(s);
  free(ids); free(sc);
  return bad;
}

int main(void) {
  int bad = 0;
  /* grid 20 x 20 with tied weights */
  {
    int64_t side = 20, n = side * side, m = 0;
    int32_t *eu = malloc(sizeof(int32_t) * 2 * n), *ev = malloc(sizeof(int32_t) * 2 * n);
    double* ew = malloc(sizeof(double) * 2 * n);
    for (int64_t i = 0; i < side; i++)
      for (int64_t j = 0; j < side; j++) {
        int64_t x = i * side + j;
        if (j + 1 < side) { eu[m] = x; ev[m] = x + 1; ew[m++] = (double)(1 + (x % 3)); }
        if (i + 1 < side) { eu[m] = x; ev[m] = x + side; ew[m++] = (double)(1 + ((x + 1) % 3)); }
      }
    bad |= run("grid", n, m, eu, ev, ew, 0);
    free(eu); free(ev); free(ew);
  }
  /* random connected graph, wide weights */
  {
    int64_t n = 300, m = 0;
    int32_t *eu = malloc(sizeof(int32_t) * 4000), *ev = malloc(sizeof(int32_t) * 4000);
    double* ew = malloc(sizeof(double) * 4000);
    unsigned s = 12345u;
    char* seen = calloc((size_t)(n * n), 1);
    for (int64_t v = 1; v < n; v++) {
      s = s * 1103515245u + 12345u;
      int64_t p = (s >> 8) % v;
      eu[m] = (int32_t)p; ev[m] = (int32_t)v; seen[p * n + v] = 1;
      ew[m++] = (double)((s >> 4) % 1000 + 1) / 37.0;
    }
    for (int k = 0; k < 1500; k++) {
      s = s * 1103515245u + 12345u; int64_t a = (s >> 8) % n;
      s = s * 1103515245u + 12345u; int64_t c = (s >> 8) % n;
      if (a == c) continue;
      int64_t x = a < c ? a : c, y = a < c ? c : a;
      if (seen[x * n + y]) continue;
      seen[x * n + y] = 1;
      eu[m] = (int32_t)x; ev[m] = (int32_t)y; ew[m++] = (double)((s >> 4) % 100000 + 1) * 1e-2;
    }
    bad |= run("random", n, m, eu, ev, ew, 0);
    free(eu); free(ev); free(ew); free(seen);
  }
  /* path (a tree: no off-tree edge) and a two-component forest */
  {
    int32_t eu[9], ev[9]; double ew[9];
    for (int i = 0; i < 9; i++) { eu[i] = i; ev[i] = i + 1; ew[i] = 1.0 + i; }
    bad |= run("path", 10, 9, eu, ev, ew, 0);
    int32_t fu[4] = {0, 1, 0, 3}, fv[4] = {1, 2, 2, 4}; double fw[4] = {1, 2, 3, 4};
    bad |= run("forest", 5, 4, fu, fv, fw, 1);
  }
  return bad;
}
"""


def test_oracle_under_asan_and_ubsan(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no gcc")
    drv = tmp_path / "drv.c"
    drv.write_text(DRIVER)
    exe = tmp_path / "drv"
    r = subprocess.run([cc, "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fsanitize=address,undefined",
                        "-fno-omit-frame-pointer", "-fno-sanitize-recover=undefined", str(drv),
                        os.path.join(ROOT, "oracle", "pdgrass_oracle.c"), "-lm", "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizers unavailable: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300, env=env)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr
    assert run.stdout.count(": ok") == 4, run.stdout
