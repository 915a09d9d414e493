"""Constants written into the kernel headers, recomputed on the host.

vegas_device.cuh holds 2^(j/64) for j = 0..63 and (ln 2)^n / n! for
n = 1..5, each the nearest double, for the FP64 path's 2^x (Tang's
table-driven method).  Here they are recomputed with 60-digit decimal
arithmetic and compared bit for bit."""
import os
import re
from decimal import Decimal, getcontext

HDR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_2010_09341_gb300", "csrc",
                   "vegas_device.cuh")


def _nearest(d: Decimal) -> float:
    return float(format(d, ".40e"))


def _array(name: str):
    txt = open(HDR).read()
    body = re.search(r"%s\[\d+\]\s*=\s*\{(.*?)\};" % name, txt, re.S).group(1)
    return [float.fromhex(v.strip()) for v in body.split(",") if v.strip()]


def test_exp2_table_is_two_to_the_j_over_64():
    getcontext().prec = 60
    tab = _array("kExp2Tab")
    assert len(tab) == 64
    for j, v in enumerate(tab):
        assert v == _nearest(Decimal(2) ** (Decimal(j) / 64)), j


def test_exp2_taylor_coefficients():
    getcontext().prec = 60
    ln2 = Decimal(2).ln()
    coef = _array("kExp2Taylor")
    assert len(coef) == 5
    f = Decimal(1)
    for n, v in enumerate(coef, start=1):
        f *= n
        assert v == _nearest(ln2 ** n / f), n
