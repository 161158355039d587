"""The generator authors' published known-answer vectors for Philox-4x32-10
(tests/golden/philox4x32_10_kat.txt, source named in the file)."""
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def published_vectors():
    """(counter words, key words, output words) per row of the fixture."""
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(v, 16) for v in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows
