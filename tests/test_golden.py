"""Stored values the paper prints (tests/golden/, each file citing its tables and equations)."""
import os

import pytest

import bench

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        out.append(line.split())
    return out


def _half_ulp(text):
    """Half a unit in the last printed digit of a decimal number."""
    d = len(text.split(".")[1]) if "." in text else 0
    return 0.5 * 10.0 ** (-d)


@pytest.mark.parametrize("row", _rows("gpp_offdiag_throughput.txt"), ids=lambda r: r[0])
def test_gpp_offdiag_flop_count_reproduces_printed_throughput(row):
    """Eq. flop_count_fullmat over the printed kernel time gives the printed PFLOP/s of the
    off-diagonal GPP rows (Si998-a/b/c), within the rounding of the printed time and rate.
    Dropping the N_G N_Sigma^2 term (1 % here), the factor 2 or swapping N_G and N_Sigma fails."""
    _, nsig, nb, ng, ne, t, pf = row
    rate = bench.gpp_offdiag_flops(int(nb), int(ne), int(nsig), int(ng)) / float(t) * 1e-15
    tol = _half_ulp(t) / float(t) + _half_ulp(pf) / float(pf)
    assert abs(rate / float(pf) - 1.0) <= tol


def test_gpp_products_are_half_the_equation_count():
    """The path runs one pair of products per (n, E): half of Eq. flop_count_fullmat's count."""
    for nb, ne, nsig, ng in [(4, 16, 512, 11075), (28224, 200, 512, 51627), (1, 1, 3, 7)]:
        assert 2 * bench.gpp_products_flops(nb, ne, nsig, ng) == bench.gpp_offdiag_flops(nb, ne, nsig, ng)
