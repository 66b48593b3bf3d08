"""The C-ABI used from plain C: a program compiled against include/*.h and
linked to libtpcfit.so checks defaults, error reporting and argument
validation (no GPU needed; without one tpcfit_create reports TPCFIT_E_NODEV)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "tpcfit.h"
#include "tpcfit_follow.h"
#include "tpcfit_rans.h"
#include "tpcfit_noalloc.h"

static int fails = 0;
#define CHECK(c) do { if (!(c)) { printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); ++fails; } } while (0)

int main(int argc, char **argv) {
  int have_gpu = argc > 1 && strcmp(argv[1], "gpu") == 0;
  tpcfit_config c;
  tpcfit_default_config(&c);
  CHECK(c.bz_tesla == 0.5f && c.chi2_max == 16.0f && c.n_rows == 152 && c.min_clusters == 10);
  CHECK(c.sort_tracks == 1 && c.res_step_y_cm == 0.01f && c.hbm_budget_bytes == (120ull << 30));
  tpcfit_follow_config f;
  tpcfit_follow_default_config(&f);
  CHECK(f.window_sigma == 4.0f && f.max_miss == 4 && f.n_sectors == 36);
  CHECK(tpcfit_rans_bound(0, 0) == 1104 && tpcfit_rans_bound(-1, 0) == -1 && tpcfit_rans_bound(10, 33) == -1);
  CHECK(strlen(tpcfit_strerror(TPCFIT_E_INVAL)) > 0 && strcmp(tpcfit_strerror(TPCFIT_OK), "ok") == 0);
  tpcfit_handle *h = 0;
  CHECK(tpcfit_create(&c, 0) == TPCFIT_E_INVAL);
  c.chi2_max = -1.0f;
  CHECK(tpcfit_create(&c, &h) == TPCFIT_E_INVAL && h == 0);
  CHECK(strlen(tpcfit_last_error_message()) > 0);
  tpcfit_default_config(&c);
  c.block_threads = 96;
  CHECK(tpcfit_create(&c, &h) == TPCFIT_E_INVAL);
  tpcfit_default_config(&c);
  CHECK(c.xrho_per_row == 0.0f && c.eloss_z_over_a == 0.0f && c.eloss_i_ev == 0.0f);
  c.xrho_per_row = 0.01f;
  c.mass_gev = 0.0f;  /* energy loss needs a mass */
  CHECK(tpcfit_create(&c, &h) == TPCFIT_E_INVAL && h == 0);
  c.mass_gev = 0.938f;
  c.eloss_i_ev = -1.0f;
  CHECK(tpcfit_create(&c, &h) == TPCFIT_E_INVAL && h == 0);
  tpcfit_default_config(&c);
  int rc = tpcfit_create(&c, &h);
  if (have_gpu) {
    CHECK(rc == TPCFIT_OK && h != 0);
    tpcfit_frame fr; memset(&fr, 0, sizeof(fr));
    tpcfit_result rs; memset(&rs, 0, sizeof(rs));
    int64_t off[1] = {0};
    fr.track_offsets = off; fr.mem = TPCFIT_MEM_HOST; rs.mem = TPCFIT_MEM_HOST;
    CHECK(tpcfit_fit(h, &fr, &rs) == TPCFIT_OK);      /* empty host frame */
    fr.n_tracks = -1;
    CHECK(tpcfit_fit(h, &fr, &rs) == TPCFIT_E_INVAL);
    CHECK(tpcfit_destroy(h) == TPCFIT_OK);
  } else {
    CHECK(rc == TPCFIT_E_NODEV && h == 0);
  }
  CHECK(tpcfit_destroy(0) == TPCFIT_E_INVAL);
  CHECK(tpcfit_fit_noalloc(0, 0, 0, 0) == TPCFIT_E_INVAL);
  printf("%s\n", fails ? "FAILED" : "ok");
  return fails != 0;
}
"""


def _build_program(tmp_path):
    from paper_2402_01205_gb300 import _build
    lib = _build.build()
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe), "-L", os.path.dirname(lib), "-Wl,-rpath," + os.path.dirname(lib),
                           "-l:" + os.path.basename(lib)])
    return exe


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_plain_c_program_without_gpu(tmp_path):
    if _has_gpu():
        pytest.skip("a GPU is present: the GPU variant of this check runs instead")
    exe = _build_program(tmp_path)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr


@pytest.mark.gpu
def test_plain_c_program_with_gpu(tmp_path):
    if not _has_gpu():
        pytest.skip("no CUDA device")
    exe = _build_program(tmp_path)
    out = subprocess.run([str(exe), "gpu"], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
