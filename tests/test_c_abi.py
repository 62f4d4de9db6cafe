"""The boundary is a plain C ABI: both headers compile as strict C99 and C11,
every declared function links against the built library, and a C program
plans a batch and reads its schedule through it (host-only calls, no GPU)."""
import os
import shutil
import subprocess

import pytest

from paper_1803_07772_gb300 import hcran

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "hcran.h"
#include "hcran_mlp.h"

/* every entry point called with NULL arguments: each rejects them with
 * HCRAN_EINVAL (or HCRAN_MLP_EINVAL) before any device work */
static int null_calls(void) {
  int bad = 0;
  bad += hcran_create(NULL, NULL, 0, NULL) != HCRAN_EINVAL;
  bad += hcran_workspace_size(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_gain_elems(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_prepare(NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_solve(NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_solve_host(NULL, NULL, NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_get(NULL, 0, NULL) != HCRAN_EINVAL;
  bad += hcran_get_summary(NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_get_phase_cycles(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_last_launch_count(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_get_schedule(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_set_schedule(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_autotune(NULL, NULL, NULL, NULL, NULL, 1) != HCRAN_EINVAL;
  bad += hcran_solve_graph(NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_warm_rows(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_warm_features(NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_solve_warm(NULL, NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_solve_noalloc(NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_set_state(NULL, NULL, 0, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_set_wait_limit(NULL, 0, -1) != HCRAN_EINVAL;
  bad += hcran_bf_workspace_size(NULL, 0, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_bruteforce(NULL, 0, NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_penalty_workspace_size(NULL, 0, NULL) != HCRAN_EINVAL;
  bad += hcran_get_stream_teams(NULL, NULL) != HCRAN_EINVAL;
  bad += hcran_penalty_solve(NULL, 0, NULL, NULL, 0.0, NULL, NULL, NULL, NULL, NULL, NULL, NULL) != HCRAN_EINVAL;
  hcran_destroy(NULL);
  bad += hcran_mlp_dense(NULL, NULL, NULL, NULL, 0, 16, 16, 0, NULL, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_tc_status(NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_create(NULL, 0, 0) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_param_count(NULL, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_get_params(NULL, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_set_params(NULL, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_get_grads(NULL, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_forward(NULL, NULL, 0, NULL, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_loss_grad(NULL, NULL, NULL, NULL, 0, 1, NULL, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_backward(NULL, NULL, 0, NULL) != HCRAN_MLP_EINVAL;
  bad += hcran_mlp_adam(NULL, 1e-3f, 0.9f, 0.999f, 1e-8f, NULL) != HCRAN_MLP_EINVAL;
  hcran_mlp_destroy(NULL);
  return bad;
}

int main(void) {
  double pmax[3] = {40.0, 1.0, 1.0}, eta[3] = {4.0, 2.0, 2.0}, pc[3] = {10.0, 1.0, 1.0}, pf[3] = {3.0, 1.0, 1.0};
  double T[2] = {0.05, 0.05}, lam[2] = {62.5, 62.5};
  hcran_config c[2];
  hcran_t h = NULL;
  int32_t cs[2] = {-1, -1};
  uint64_t ws = 0;
  int i, rc;
  for (i = 0; i < 2; i++) {
    c[i].M = 3; c[i].N = 16 + 16 * i; c[i].K = 6; c[i].Ks = 2; c[i].l = 2;
    c[i].pmax = pmax; c[i].eta = eta; c[i].Pc = pc; c[i].Pf = pf;
    c[i].Bn_hz = 180e3; c[i].N0_w_per_hz = 3.98e-21;
    c[i].T_s = T; c[i].lambda_pps = lam; c[i].zbar_bits = 1024.0; c[i].w = NULL;
  }
  rc = null_calls();
  if (rc != 0) {
    printf("%d entry points accepted NULL\n", rc);
    return 10;
  }
  rc = hcran_create(&h, c, 2, NULL);
  if (rc != HCRAN_OK) return 11;
  if (hcran_workspace_size(h, &ws) != HCRAN_OK || ws == 0) return 12;
  if (hcran_get_schedule(h, cs) != HCRAN_OK) return 13;
  if (hcran_get_schedule(h, NULL) != HCRAN_EINVAL) return 14;
  printf("%d %d %llu\n", cs[0], cs[1], (unsigned long long)ws);
  hcran_destroy(h);
  return 0;
}
"""


@pytest.mark.parametrize("std", ["c99", "c11"])
def test_headers_compile_as_c_and_link(tmp_path, std):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = hcran.load()
    so = lib._name
    src = tmp_path / "use_abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_abi"
    subprocess.run([cc, "-std=" + std, "-pedantic", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), so, "-Wl,-rpath," + os.path.dirname(so),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    cs0, cs1, ws = out.stdout.split()
    assert 1 <= int(cs0) <= 8 and 1 <= int(cs1) <= 8 and int(ws) > 0
