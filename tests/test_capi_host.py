"""Host-side checks of the C-ABI library (no GPU needed).

* The library builds for sm_103a and loads; it exports every entry point that
  include/pic.h declares.
* The ctypes mirror of every struct has the size and field offsets the C compiler
  gives the header.
* pic_create rejects invalid configurations before touching the GPU, and reports why.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2404_10270_gb300 import build as B
from paper_2404_10270_gb300 import capi
from paper_2404_10270_gb300 import workloads as W
from tests.helpers import ROOT

HEADER = os.path.join(ROOT, "include", "pic.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return capi.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"PIC_API\s+[\w\s\*]*?\b(pic_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pic_create", "pic_load_particles", "pic_step", "pic_moments", "pic_destroy",
              "pic_get_particles", "pic_last_error"):
        assert n in names
    assert set(names) == set(capi.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", capi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pic_\w+)", out))
    for n in declared_functions():
        assert n in exported, n
        assert hasattr(L, n)


def _c_layout(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "pic.h"
#define P(T, f) printf(#T "." #f " %zu\\n", offsetof(T, f));
int main(void) {
  printf("pic_species %zu\\n", sizeof(pic_species));
  printf("pic_process %zu\\n", sizeof(pic_process));
  printf("pic_instance %zu\\n", sizeof(pic_instance));
  printf("pic_config %zu\\n", sizeof(pic_config));
  printf("pic_moments_out %zu\\n", sizeof(pic_moments_out));
  P(pic_instance, dx) P(pic_instance, B) P(pic_instance, sp) P(pic_instance, nproc)
  P(pic_instance, proc) P(pic_instance, seed) P(pic_config, inst) P(pic_config, cuda_stream)
  P(pic_moments_out, wall_count) P(pic_moments_out, wall_energy) P(pic_moments_out, collisions)
  P(pic_moments_out, kinetic) P(pic_species, capacity) P(pic_process, nu)
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return dict(line.split() for line in out.strip().splitlines())


def test_ctypes_layout_matches_header(tmp_path):
    c = {k: int(v) for k, v in _c_layout(tmp_path).items()}
    assert C.sizeof(capi.pic_species) == c["pic_species"]
    assert C.sizeof(capi.pic_process) == c["pic_process"]
    assert C.sizeof(capi.pic_instance) == c["pic_instance"]
    assert C.sizeof(capi.pic_config) == c["pic_config"]
    assert C.sizeof(capi.pic_moments_out) == c["pic_moments_out"]
    for key, v in c.items():
        if "." not in key:
            continue
        struct, field = key.split(".")
        assert getattr(getattr(capi, struct), field).offset == v, key


def _create(L, inst_list, precision=capi.FP32, block=0, sort_interval=0):
    arr = (capi.pic_instance * len(inst_list))(*inst_list)
    cfg = capi.pic_config()
    cfg.n_instances = len(inst_list)
    cfg.precision = precision
    cfg.sort_interval = sort_interval
    cfg.block = block
    cfg.inst = arr
    h = C.c_void_p()
    rc = L.pic_create(C.byref(cfg), C.byref(h))
    return rc, h


@pytest.mark.parametrize("mutate,needle", [
    (lambda I: setattr(I, "ncells", 0), "ncells"),
    (lambda I: setattr(I, "dx", -1.0), "dx"),
    (lambda I: setattr(I, "nspecies", 5), "nspecies"),
    (lambda I: setattr(I, "bc", W.BC_PERIODIC), "Poisson"),
    (lambda I: setattr(I.proc[0], "species", 7), "process species"),
    (lambda I: setattr(I, "m_neutral", 2.0), "elastic"),
    (lambda I: setattr(I.sp[1], "weight", 0.003), "integer multiples"),
])
def test_create_rejects_invalid_instances(L, mutate, needle):
    I = capi.instance_struct(W.bounded_small(ncells=16, ppc=4))
    mutate(I)
    rc, h = _create(L, [I])
    assert rc == -1 and not h.value
    assert needle in L.pic_last_error(None).decode()


def test_create_rejects_invalid_neutral_targets(L):
    base = W.ionization_case(ncells=16, ppc=4)
    for mutate, needle in ((lambda I: setattr(I.sp[2], "charge", 1.0), "charge 0"),
                           (lambda I: setattr(I, "nref", 0), "nref"),
                           (lambda I: setattr(I, "target", 9), "target")):
        I = capi.instance_struct(base)
        mutate(I)
        rc, h = _create(L, [I], sort_interval=base.sort_interval)
        assert rc == -1 and not h.value
        assert needle in L.pic_last_error(None).decode()
    # the target's nstep must equal the (fixed) sort interval
    I = capi.instance_struct(base)
    for si in (base.sort_interval + 1, -1):
        rc, h = _create(L, [I], sort_interval=si)
        assert rc == -1 and "sort interval" in L.pic_last_error(None).decode()


def test_create_rejects_invalid_config(L):
    I = capi.instance_struct(W.bounded_small(ncells=16, ppc=4))
    for kw in (dict(precision=7), dict(block=100), dict(sort_interval=-2)):
        rc, h = _create(L, [I], **kw)
        assert rc == -1 and not h.value
    assert L.pic_create(None, None) == -1


def test_null_safe_calls(L):
    assert L.pic_destroy(None) == 0
    assert L.pic_step(None, 1) == -1
    assert L.pic_philox(1, None, None, 0, 0, None) == 0
