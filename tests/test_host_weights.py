"""The library's host weight generator (C++, long double) against the oracle's
weight tables (exact rationals or 60-digit mpmath), through the C ABI on the CPU:
the two are written independently, so a wrong node, index or window in either
fails here. sdc_scheme_weights needs no device."""

import numpy as np
import pytest

from oracle.weights import mrsdc_weights

CASES = [("equi_noleft", 3, 2, 0), ("equi_noleft", 5, 8, 8), ("equi_noleft", 5, 8, 0), ("equi_noleft", 4, 3, 3),
         ("radau_right", 3, 4, 0), ("radau_right", 4, 40, 0), ("radau_right", 1, 5, 0), ("lobatto", 3, 20, 0),
         ("lobatto", 4, 6, 2), ("lobatto", 2, 1, 0)]


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03581_gb300 import build

    build.build()


@pytest.mark.parametrize("nodes,M,P,w", CASES)
def test_host_weights_match_the_oracle(lib, nodes, M, P, w):
    from paper_1707_03581_gb300.binding import scheme_weights

    got = scheme_weights(nodes, M, P, w)
    ref = mrsdc_weights(nodes, M, P, w)
    for key in ("c", "emb", "S", "Shat", "Stil", "Semb"):
        a = np.asarray(got[key], dtype=np.float64)
        b = np.asarray(ref[key], dtype=np.float64).reshape(a.shape)
        scale = max(np.abs(b).max(), 1e-300)
        assert np.abs(a - b).max() <= 4e-15 * scale, (key, np.abs(a - b).max(), scale)


def test_host_weights_refuse_what_the_scheme_refuses(lib):
    from paper_1707_03581_gb300.binding import SdcError, scheme_weights

    for args in (("lobatto", 1, 4, 0), ("equi_noleft", 3, 65, 0), ("equi_noleft", 3, 4, 5), ("radau_right", 0, 2, 0)):
        with pytest.raises(SdcError):
            scheme_weights(*args)
