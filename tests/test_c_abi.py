"""The C ABI from plain C: include/tho.h compiles as C99 with warnings as
errors, and a C program linked against libtho.so (no Python, no torch) gets
the host-side answers -- argument and shape errors before any CUDA call, status
strings, the autotuner's cache key and cache file."""
import os
import subprocess

import pytest

from paper_2602_14449_gb300 import build as tho_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "tho.h"

static int fails = 0;
#define CHECK(c) do { if (!(c)) { printf("FAIL line %d: %s\n", __LINE__, #c); ++fails; } } while (0)

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  const char* cache = argv[1];
  tho_desc_t d = {4096, 16, 4, THO_F64, THO_PREC_FP64, 0};
  tho_plan_t plan = NULL;
  tho_desc_t bad = d;
  bad.k0 = 4093;                                   /* k0 + k > n */
  CHECK(tho_plan(&bad, 1, &plan) == THO_ERR_SHAPE && plan == NULL);
  bad = d; bad.k = THO_MAX_K + 1;
  CHECK(tho_plan(&bad, 1, &plan) == THO_ERR_UNSUPPORTED);
  CHECK(tho_plan(NULL, 1, &plan) == THO_ERR_ARG);
  tho_tuning_t t = {100, 0, 0};                    /* not a leaf height */
  CHECK(tho_plan_tuned(&d, 1, &t, &plan) == THO_ERR_ARG);
  CHECK(tho_orth(NULL, NULL, 0, NULL, 0, NULL, 0, NULL, NULL, NULL) == THO_ERR_ARG);
  CHECK(tho_plan_destroy(NULL) == THO_OK);
  CHECK(strcmp(tho_status_string(THO_OK), "success") == 0);
  CHECK(strcmp(tho_phase_name(3), "leaf") == 0 && tho_phase_name(THO_NUM_PHASES) == NULL);
  char key[256];
  CHECK(tho_tune_key(&d, 1, "gpu", key, sizeof key) == THO_OK);
  CHECK(strcmp(key, "gpu|f64|fp64|f0|q48:16:4") == 0);
  tho_tuning_t put = {128, 303, 0}, got = {0, 0, 0};
  double ms = 0.0;
  int32_t found = 0;
  CHECK(tho_tune_cache_put(cache, key, &put, 1.5) == THO_OK);
  CHECK(tho_tune_cache_get(cache, key, &got, &ms, &found) == THO_OK);
  CHECK(found == 1 && got.leaf_rows == 128 && got.split_chunks == 303 && got.balance == 0 && ms == 1.5);
  printf("%s\n", fails ? "failed" : "ok");
  return fails != 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    tho_build.build()
    return os.path.dirname(tho_build.LIB)


def test_header_compiles_as_c99_and_the_library_answers_from_c(libdir, tmp_path):
    src = tmp_path / "use_tho.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_tho"
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                         str(src), "-o", str(exe), "-L", libdir, "-ltho", f"-Wl,-rpath,{libdir}"],
                        capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe), str(tmp_path / "cache.jsonl")], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
