"""The C-ABI library loads and exports every entry point include/cdfci.h declares,
and the Python binding's structures have the C layout (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cdfci.h")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_04483_gb300 import api
    return api


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cdfci_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(built):
    names = declared_functions()
    assert "cdfci_create" in names and "cdfci_step" in names
    L = built.lib()
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/cdfci.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", built.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (cdfci_\w+)", out))
    assert set(names) == exported, (set(names) ^ exported)


def test_struct_layouts_match_header(built, tmp_path):
    ck = built.cdfci_checkpoint_header
    ck_lines = "\n".join(f"  F(cdfci_checkpoint_header, {f})" for f, _ in ck._fields_)
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "cdfci.h"
#define F(T, f) printf("%s.%s %zu\\n", #T, #f, offsetof(T, f));
int main(void) {
  printf("cdfci_params %zu\\n", sizeof(cdfci_params));
  printf("cdfci_stats %zu\\n", sizeof(cdfci_stats));
  printf("cdfci_tune_report %zu\\n", sizeof(cdfci_tune_report));
  F(cdfci_params, z_threshold) F(cdfci_params, ref_alpha) F(cdfci_params, block_threads)
  F(cdfci_params, deterministic) F(cdfci_params, cuda_stream)
  F(cdfci_stats, energy) F(cdfci_stats, nnz_c) F(cdfci_stats, load) F(cdfci_stats, status) F(cdfci_stats, converged) F(cdfci_stats, reduced_iterations)
  F(cdfci_stats, grid_blocks) F(cdfci_stats, grid_wide)
  F(cdfci_tune_report, chosen) F(cdfci_tune_report, m) F(cdfci_tune_report, grid_blocks) F(cdfci_tune_report, iterations) F(cdfci_tune_report, seconds)
  F(cdfci_tune_report, energy_drop) F(cdfci_tune_report, score)
  printf("cdfci_checkpoint_header %zu\\n", sizeof(cdfci_checkpoint_header));
  printf("cdfci_optorb_params %zu\\n", sizeof(cdfci_optorb_params));
  F(cdfci_optorb_params, inner_iterations) F(cdfci_optorb_params, fci)
  F(cdfci_params, num_states) F(cdfci_params, z_threshold_search) F(cdfci_params, max_memory)
  F(cdfci_stats, z_threshold)
""" + ck_lines + """
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    vals = dict(l.split() for l in lines if l.strip())
    P, S, R = built.cdfci_params, built.cdfci_stats, built.cdfci_tune_report
    assert int(vals["cdfci_params"]) == ctypes.sizeof(P)
    assert int(vals["cdfci_stats"]) == ctypes.sizeof(S)
    assert int(vals["cdfci_tune_report"]) == ctypes.sizeof(R)
    assert int(vals["cdfci_checkpoint_header"]) == ctypes.sizeof(ck)
    assert int(vals["cdfci_optorb_params"]) == ctypes.sizeof(built.cdfci_optorb_params)
    for k, v in vals.items():
        if "." in k:
            t, f = k.split(".")
            cls = {"cdfci_params": P, "cdfci_stats": S, "cdfci_tune_report": R, "cdfci_checkpoint_header": ck,
                   "cdfci_optorb_params": built.cdfci_optorb_params}[t]
            assert getattr(cls, f).offset == int(v), k


def test_defaults_and_errors_without_gpu(built):
    p = built.cdfci_default_params()
    assert p.num_coordinates == 1 and abs(p.max_load - 0.79) < 1e-15 and p.z_threshold == 0.0
    assert p.deterministic == 1
    # argument errors are reported before any device work
    import numpy as np
    h = np.zeros((4, 4))
    g = np.zeros((4, 4, 4, 4))
    with pytest.raises(built.CdfciError) as e:
        built.cdfci_create(h, g, 70, 1, 1)
    assert e.value.code == -1
    with pytest.raises(built.CdfciError) as e:
        built.cdfci_create(h, g, 4, 5, 1)
    assert e.value.code == -1
    bad_ref = built.cdfci_default_params(ref_alpha=0b111, ref_beta=0b1)
    with pytest.raises(built.CdfciError) as e:
        built.cdfci_create(h, g, 4, 2, 1, bad_ref)
    assert e.value.code == -1


def test_new_entry_points_check_arguments_without_gpu(built):
    """integral_symmetry, the k-space lattice's shape and parameters, and NULL handles are
    rejected with CDFCI_ERR_ARG before any device work."""
    import numpy as np
    h = np.zeros((4, 4))
    g = np.zeros((4, 4, 4, 4))
    with pytest.raises(built.CdfciError) as e:
        built.cdfci_create(h, g, 4, 2, 1, built.cdfci_default_params(integral_symmetry=3))
    assert e.value.code == -1
    assert built.cdfci_default_params().integral_symmetry == 8
    for shape, t, U in [([], 1.0, 4.0), ([0, 4], 1.0, 4.0), ([9, 8], 1.0, 4.0), ([2] * 9, 1.0, 4.0),
                        ([4, 4], float("inf"), 4.0), ([4, 4], 1.0, float("nan"))]:
        with pytest.raises(built.CdfciError) as e:
            built.cdfci_create_hubbard_k(shape, t, U, 2, 2)
        assert e.value.code == -1, (shape, t, U)
    L = built.lib()
    assert L.cdfci_get_entry(None, None, None, None) == -1
    assert L.cdfci_get_diagonal(None, None, None) == -1
    assert L.cdfci_time_kernels(None, 1, None, 0, None) == -1
    assert L.cdfci_set_initial_degenerate(None, 0.0, 0, None, None) == -1


def test_degenerate_set_requires_a_capacity_with_a_buffer(built):
    """With a keys buffer, cap <= 0 is an argument error (no default capacity that could overrun a
    smaller buffer); without one, cap <= 0 only asks for the count."""
    import ctypes
    import numpy as np
    L = built.lib()
    eps = np.array([-2.0, 0.0, 0.0, 0.0, 0.0, 2.0])        # 1 + 4 degenerate levels + 1
    n = ctypes.c_int64(-1)
    keys = np.zeros((2, 2), dtype=np.uint64)
    assert L.cdfci_degenerate_set(eps.ctypes.data, 6, 2, 2, 0.0, 0, keys.ctypes.data, ctypes.byref(n)) == -1
    assert (keys == 0).all()
    assert L.cdfci_degenerate_set(eps.ctypes.data, 6, 2, 2, 0.0, 0, None, ctypes.byref(n)) == 0
    assert n.value == 16                                     # 4 choices per spin


def test_noalloc_source_allocates_nothing():
    """The allocation-free entry point's translation unit calls no allocating CUDA routine."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2605_04483_gb300", "csrc", "cdfci_noalloc.cu")).read()
    code = re.sub(r"/\*.*?\*/", "", re.sub(r"//[^\n]*", "", src), flags=re.S)
    for call in ("cudaMalloc", "cudaMallocAsync", "cudaMallocManaged", "cudaMallocHost", "cudaHostAlloc",
                 "cudaFree", "cuMemAlloc", "malloc(", "new "):
        assert call not in code, call
    assert "static __device__ __align__(256)" in code and "cudaGetSymbolAddress" in code
