"""The counter-based generator of the genetic search, against its published vectors."""
import os

from tests._philox import philox4x32_10


def test_reference_reproduces_published_vectors():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert philox4x32_10(w[0:4], w[4:6]) == w[6:10]
        n += 1
    assert n == 3
