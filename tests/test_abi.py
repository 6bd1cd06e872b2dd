"""The C ABI: the library loads, exports every entry point the header declares,
and the Python mirrors of its structs match the C layout.  No compute calls
(no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def mt():
    import paper_1710_05785_b300 as m
    from paper_1710_05785_b300 import build as b
    b.build()
    return m


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for mo in re.finditer(r"\b(maiter_\w+)\s*\(", text):
            names.add(mo.group(1))
    return sorted(names)


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ["maiter_graph_create", "maiter_run", "maiter_get_state"]:
        assert core in names


def test_library_exports_every_declared_symbol(mt):
    L = mt.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", mt.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(declared_functions()) <= exported
    # nothing but the C ABI leaks out of the shared object
    assert all(s.startswith("maiter_") for s in exported), sorted(exported)[:10]


def test_version_and_defaults_without_gpu(mt):
    assert "sm_103a" in mt.version()
    p = mt.params_default()
    assert p.op == mt.OP_SUM_F64 and p.damping == 0.8 and p.eps == 1e-8
    assert p.source == -1 and p.max_rounds == 1000000


def test_struct_layout_matches_c(mt, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "maiter.h"
#define F(s, f) printf("%s.%s %zu\n", #s, #f, offsetof(s, f))
int main(void) {
  printf("run_params %zu\n", sizeof(maiter_run_params));
  printf("stats %zu\n", sizeof(maiter_stats));
  F(maiter_run_params, coef); F(maiter_run_params, damping); F(maiter_run_params, v0);
  F(maiter_run_params, delta0); F(maiter_run_params, source); F(maiter_run_params, threshold);
  F(maiter_run_params, top_frac); F(maiter_run_params, eps); F(maiter_run_params, max_rounds);
  F(maiter_run_params, timeout_ms); F(maiter_run_params, stream);
  F(maiter_stats, residual); F(maiter_stats, elapsed_ms); F(maiter_stats, status);
  F(maiter_stats, converged); F(maiter_stats, kernel_launches); F(maiter_stats, push_ms);
  F(maiter_stats, scan_launches); F(maiter_run_params, flags);
  F(maiter_run_params, mixed_switch);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = dict(l.rsplit(" ", 1) for l in lines if l)
    assert int(c["run_params"]) == ctypes.sizeof(mt.RunParams)
    assert int(c["stats"]) == ctypes.sizeof(mt.Stats)
    for key, val in c.items():
        if "." in key:
            s, f = key.split(".")
            cls = mt.RunParams if s == "maiter_run_params" else mt.Stats
            assert getattr(cls, f).offset == int(val), key


def test_binding_holds_no_fallback():
    # the binding never imports the oracle or computes results itself
    src = open(os.path.join(ROOT, "paper_1710_05785_b300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_oracle_and_cuda_path_share_no_code():
    cu_dir = os.path.join(ROOT, "paper_1710_05785_b300", "csrc")
    for f in os.listdir(cu_dir):
        text = open(os.path.join(cu_dir, f)).read()
        assert "oracle" not in text.lower(), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".py")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1710_05785_b300" not in text and "csrc" not in text, f


def test_probe_rejects_bad_arguments_before_any_device_work(mt):
    for kind, lg in [(4, 20), (-1, 20), (mt.PROBE_RED_F32, 9), (mt.PROBE_LOAD_32, 29)]:
        with pytest.raises(mt.MaiterError) as ei:
            mt.probe_random_rate(kind, lg)
        assert ei.value.status == mt.ERR_INVALID_ARG
