"""FCIDUMP ingestion (cdfci_fcidump_header / cdfci_fcidump_read, host code of the library; Sec.
"Example Usage": the molecular Hamiltonian read from an FCIDUMP file with a truncation threshold for
small integral values).  No GPU needed."""
import numpy as np
import pytest

from paper_2605_04483_gb300 import inputs


@pytest.fixture(scope="module")
def api():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_04483_gb300 import api as a
    return a


@pytest.mark.parametrize("fortran", [False, True])
def test_round_trip_is_bit_exact(api, tmp_path, fortran):
    w = inputs.ab_initio(8, 3, 2, seed=3)
    p = tmp_path / "x.FCIDUMP"
    inputs.write_fcidump(str(p), w, e_core=9.8765432109876, fortran=fortran)
    r = api.cdfci_fcidump_read(str(p))
    assert (r["N"], r["n_alpha"], r["n_beta"]) == (8, 3, 2)
    assert np.array_equal(r["h"], w.h) and np.array_equal(r["g"], w.g)
    assert r["e_core"] == 9.8765432109876


def test_threshold_neglects_small_values_only(api, tmp_path):
    w = inputs.ab_initio(7, 2, 2, seed=4)
    p = tmp_path / "t.FCIDUMP"
    inputs.write_fcidump(str(p), w, e_core=-1.5)
    thr = 2e-3
    r = api.cdfci_fcidump_read(str(p), threshold=thr)
    assert np.array_equal(r["g"], np.where(np.abs(w.g) < thr, 0.0, w.g))
    assert np.array_equal(r["h"], np.where(np.abs(w.h) < thr, 0.0, w.h))
    assert 0 < np.count_nonzero(np.abs(w.g) < thr) < w.g.size - np.count_nonzero(w.g == 0)
    assert r["e_core"] == -1.5                       # a constant, never truncated


def test_header_variants_and_index_patterns(api, tmp_path):
    # lower case, "/" as the end, spin polarisation, orbital-energy lines skipped,
    # one integral standing for its 8 images, h symmetric
    text = """ &fci norb = 3, nelec=3, ms2=1,
  orbsym=1,1,1, isym=1
 /
  0.5 1 2 3 1
 -1.25D+00 2 1 0 0
  0.75 3 3 3 3
  -0.4 2 0 0 0
  2.0 0 0 0 0
"""
    p = tmp_path / "h.FCIDUMP"
    p.write_text(text)
    assert api.cdfci_fcidump_header(str(p)) == (3, 3, 1)
    r = api.cdfci_fcidump_read(str(p))
    assert (r["n_alpha"], r["n_beta"], r["e_core"]) == (2, 1, 2.0)
    g = r["g"]
    for (a, b, c, d) in [(0, 1, 2, 0), (1, 0, 2, 0), (0, 1, 0, 2), (1, 0, 0, 2),
                         (2, 0, 0, 1), (0, 2, 0, 1), (2, 0, 1, 0), (0, 2, 1, 0)]:
        assert g[a, b, c, d] == 0.5
    assert g[2, 2, 2, 2] == 0.75 and np.count_nonzero(g) == 9
    assert r["h"][1, 0] == r["h"][0, 1] == -1.25 and np.count_nonzero(r["h"]) == 2


@pytest.mark.parametrize("body,code", [
    ("1.0 1 2 3\n", -1),                  # a short line
    ("1.0 1 2 4 1\n", -1),                # an index beyond NORB
    ("1.0 1 0 2 0\n", -1),                # no valid pattern
    ("nan 1 1 1 1\n", -2),                # not finite
])
def test_malformed_files_are_rejected(api, tmp_path, body, code):
    p = tmp_path / "bad.FCIDUMP"
    p.write_text(" &FCI NORB=3,NELEC=2,MS2=0 &END\n" + body)
    with pytest.raises(api.CdfciError) as e:
        api.cdfci_fcidump_read(str(p))
    assert e.value.code == code


def test_missing_file_and_bad_header(api, tmp_path):
    with pytest.raises(api.CdfciError):
        api.cdfci_fcidump_header(str(tmp_path / "absent"))
    p = tmp_path / "nohdr.FCIDUMP"
    p.write_text("1.0 1 1 1 1\n")
    with pytest.raises(api.CdfciError):
        api.cdfci_fcidump_header(str(p))
    p.write_text(" &FCI NORB=2,NELEC=5,MS2=0 &END\n")      # more electrons than spin-orbitals
    with pytest.raises(api.CdfciError):
        api.cdfci_fcidump_header(str(p))
