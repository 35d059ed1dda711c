"""The C ABI used from plain C: include/emugemm.h compiles as strict C99,
a C program that takes the address of every declared entry point links
against the in-tree library (so every name resolves unmangled), and its
host-side checks run without a GPU (argument validation, status strings,
workspace sizes, handle creation reporting EMU_ERR_CUDA on a machine with
no GPU)."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "emugemm.h")

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")


def declared_functions():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(emu_[A-Za-z0-9_]+)\s*\(", src)))


PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "emugemm.h"

static void (*const entry[])(void) = { %(entries)s };

int main(void) {
  size_t bytes = 0;
  emu_handle_t h = NULL;
  emu_status_t s;
  int bad = 0;
  if (sizeof(entry) / sizeof(entry[0]) != %(count)d) bad |= 1;
  /* argument checks that need no device */
  if (emu_dgemm(NULL, EMU_ROW_MAJOR, 4, 4, 4, 1.0, NULL, 4, NULL, 4, 0.0, NULL, 4, EMU_SCHEME_I, 3, NULL) !=
      EMU_ERR_INVALID_ARG) bad |= 2;
  if (emu_workspace_size(EMU_SCHEME_I, 100, 100, 100, 8, 0, &bytes) != EMU_OK || bytes == 0) bad |= 4;
  if (emu_workspace_size(EMU_SCHEME_I, 10, 10, 10, EMU_P_MAX + 1, 0, &bytes) != EMU_ERR_UNSUPPORTED) bad |= 8;
  if (strcmp(emu_status_string(EMU_ERR_TIMEOUT), "EMU_ERR_TIMEOUT") != 0) bad |= 16;
  s = emu_create(&h, 0);
  if (s == EMU_OK) {
    emu_destroy(h);
  } else if (s != EMU_ERR_CUDA) {
    bad |= 32;
  }
  printf("create=%%d bad=%%d\n", (int)s, bad);
  return bad;
}
"""


def test_header_is_strict_c99():
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c",
                    HEADER], check=True)


def test_c_program_links_every_entry_point(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    libdir = os.path.join(ROOT, "paper_2606_25453_gb300", "_build")
    names = declared_functions()
    assert len(names) >= 35
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM % {"entries": ", ".join("(void (*)(void))%s" % n for n in names), "count": len(names)})
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), "-L", libdir, "-lemugemm", "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "bad=0" in r.stdout
