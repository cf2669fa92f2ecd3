"""The C-ABI library loads and exports every function include/rec.h declares
(no GPU needed: nothing is launched), and its host-side transport scalars are
bit-identical to the oracle's (they define the bytes the transport consumes)."""
import os
import re

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b((?:rec|lya)_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2312_11448_gb300 import rec
    L = rec.lib()
    names = _declared()
    assert {"rec_init", "lya_transport", "rec_step", "rec_step_adjoint", "rec_free"} <= set(names)
    for name in names:
        assert hasattr(L, name), name


@pytest.mark.parametrize("n,z", [(8, 1800.0), (32, 1600.0), (128, 1234.5678), (256, 1100.0), (512, 600.0)])
def test_transport_scalars_bit_identical_to_oracle(n, z):
    from paper_2312_11448_gb300 import rec
    assert rec.transport_params(n, z) == O.transport_params(O.default_cosmo(), n, z)


def test_invalid_params_rejected_without_gpu():
    from paper_2312_11448_gb300 import rec
    with pytest.raises(rec.RecError):
        rec.transport_params(16, -5.0)
    with pytest.raises(rec.RecError):
        rec.transport_params(16, 1000.0, h=-1.0)
