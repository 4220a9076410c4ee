"""Writes the exact triangle counts N_T (eq. NT) of a shell set on a grid,
computed by the FP64 oracle (oracle.bispectrum.Counter: per-mode rounded
convolution of shell indicators), as a text fixture for the GPU tests.

Usage: python tests/golden/make_triangle_counts.py N first step width S out.txt
The default fixture is the bispectrum workload's shells on its 360^3 grid:
    python tests/golden/make_triangle_counts.py 360 3 3 3 37 \
        tests/golden/triangle_counts_360_s37.txt
Every triple a >= b >= c with N_T > 0 is listed as "a b c N_T".  With
3 n_max < N the counts depend only on the shells, so the 27 innermost shells'
triangles are also those of the 27-shell sets on 256^3 and 384^3 grids.
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle.bispectrum import Counter  # noqa: E402


def main(argv):
    N, first, step, width, S = (int(v) for v in argv[:5])
    out = argv[5]
    t0 = time.time()
    counter = Counter(N, (first, step, width, S))
    rows = []
    for b in range(S):
        for c in range(b + 1):
            nt = counter.counts_for_pair(b, c, keep=False)
            for a in range(b, S):
                if nt[a] > 0:
                    rows.append((a, b, c, int(nt[a])))
        print(f"b={b} done, {time.time() - t0:.0f} s", flush=True)
    rows.sort()
    with open(out, "w") as f:
        f.write(f"# exact N_T (oracle.bispectrum.Counter), N={N}, shells first={first} step={step} "
                f"width={width} S={S} (integer k_f units); a >= b >= c, N_T > 0\n")
        for r in rows:
            f.write("%d %d %d %d\n" % r)
    print(len(rows), "triangles")


if __name__ == "__main__":
    main(sys.argv[1:])
