"""The library's ESDIRK tableaus (host code, no GPU needed) against the oracle's."""
import numpy as np
import pytest

from oracle import esdirk


@pytest.mark.parametrize("order,ref", [(2, esdirk.esdirk2()), (3, esdirk.esdirk3())])
def test_library_tableau_matches_oracle(order, ref):
    from paper_1910_03693_gb300 import build as B
    B.build()
    from paper_1910_03693_gb300 import esdirk_tableau
    A, b = esdirk_tableau(order)
    assert np.allclose(np.array(A), np.array(ref.A), atol=1e-15, rtol=0)
    assert np.allclose(np.array(b), np.array(ref.b), atol=1e-15, rtol=0)
