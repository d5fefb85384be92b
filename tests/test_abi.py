"""Host-side checks of the C ABI (no GPU): the library loads, exports every
entry point include/afqmc.h declares, and rejects bad parameters before any
device work."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "afqmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(afqmc_[a-z_A-Z]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2609_14668_b300 import build
    build.build()
    lib = ctypes.CDLL(build.LIB)
    syms = declared_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    import paper_2609_14668_b300 as pkg
    assert sorted(pkg.EXPORTED) == declared_symbols()
    for s in declared_symbols():
        assert callable(getattr(pkg, s))


@pytest.mark.parametrize("field,value,msg", [
    ("L1", 0, "L1"), ("beta", -1.0, "beta"), ("dtau", 0.0, "dtau"), ("n_stab", 7, "n_stab"),
    ("n_delay", 0, "n_delay"), ("theta1", 1.5, "twist"), ("theta2", -0.25, "twist"), ("hs_channel", 2, "charge channel"), ("hs_channel", -1, "hs_channel"),
    ("precision", 4, "precision"), ("precision", 5, "precision"), ("precision", 8, "precision"), ("U", -1.0, "U"),
])
def test_invalid_parameters_rejected_on_host(field, value, msg):
    import paper_2609_14668_b300 as pkg
    p = pkg.make_params(L=3, beta=3.0, dtau=0.1, U=3.73, n_delay=4, n_stab=10)
    setattr(p, field, value)
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_create(p)
    assert e.value.code == 1
    assert msg.split()[0].lower() in str(e.value).lower()


def test_beta_not_multiple_of_dtau():
    import paper_2609_14668_b300 as pkg
    p = pkg.make_params(L=3, beta=3.05, dtau=0.1, U=3.73, n_delay=4, n_stab=1)
    with pytest.raises(pkg.AfqmcError) as e:
        pkg.afqmc_create(p)
    assert e.value.code == 1


def test_kernel_families_match_header():
    """The binding's family names and timing struct follow the header's enum."""
    import ctypes
    import paper_2609_14668_b300 as pkg
    src = open(os.path.join(ROOT, "include", "afqmc.h")).read()
    fams = dict((k, int(v)) for k, v in re.findall(r"\bAFQMC_K_([A-Z]+)\s*=\s*(\d+)", src))
    count = fams.pop("COUNT")
    assert count == len(pkg.KERNEL_FAMILIES) == len(fams)
    assert sorted(fams.values()) == list(range(count))
    names = {"QRAUX": "qr_aux"}
    for k, v in fams.items():
        assert pkg.KERNEL_FAMILIES[v] == names.get(k, k.lower())
    assert ctypes.sizeof(pkg.afqmc_timing) == 16 * count
    assert pkg.TIMING_ALL == (1 << count) - 1
