"""Host checks of the index scheme of the compile-time shared-memory FFT
(csrc/fkp_fft.cuh), restated here in Python: the radix order, the Stockham
stages (butterfly j of a radix-R stage after stages of product ns reads
x[j + r n/R], multiplies by w^(r k n/(ns R)) with k = j mod ns, and writes
y[(j/ns) ns R + k + r ns]) reproduce the DFT, and for the sizes whose last
stage the y-pass takes from registers, the outputs a thread's last-stage
butterflies produce are exactly its k_y = y + i NT/P."""
import numpy as np
import pytest


def radices(n):
    """The radix order of the kernels: 8s first, then 4, 2, 5, 3."""
    out = []
    for r in (8, 4, 2, 5, 3):
        while n % r == 0:
            out.append(r)
            n //= r
    assert n == 1
    return out


def stockham(x, sign=-1):
    n = x.size
    ns = 1
    a = x.astype(np.complex128)
    for R in radices(n):
        nb = n // R
        b = np.empty_like(a)
        for j in range(nb):
            k = j % ns
            v = np.array([a[j + r * nb] for r in range(R)])
            tw = np.exp(sign * 2j * np.pi * np.arange(R) * k * (n // (ns * R)) / n)
            v = v * tw
            d = np.array([np.sum(v * np.exp(sign * 2j * np.pi * np.arange(R) * q / R)) for q in range(R)])
            base = (j // ns) * ns * R + k
            for r in range(R):
                b[base + r * ns] = d[r]
        a = b
        ns *= R
    return a


@pytest.mark.parametrize("n", [8, 12, 48, 60, 64, 90, 128, 360, 384, 512])
def test_stockham_stages_are_the_dft(n):
    x = np.random.default_rng(n).standard_normal(n) + 1j * np.random.default_rng(n + 1).standard_normal(n)
    assert np.allclose(stockham(x), np.fft.fft(x), atol=1e-9 * n)
    assert np.allclose(stockham(x, +1), np.fft.ifft(x) * n, atol=1e-9 * n)


def fusable(n, P, NT):
    rs = radices(n)
    return len(rs) >= 2 and (n // rs[-1]) % (NT // P) == 0


@pytest.mark.parametrize("n", [128, 256, 384, 512])
@pytest.mark.parametrize("NT", [256, 512])
def test_last_stage_outputs_are_the_threads_runs(n, NT):
    """Thread (p, y) of a (P, NT/P) block takes butterflies j = j0 + y,
    j0 = 0, NT/P, ... < n/R of the last stage (R its radix); those write
    j + r n/R.  Their union is {y + i NT/P}: the y-pass's run of k_y for
    that thread, each once."""
    P = 8
    JT = NT // P
    assert fusable(n, P, NT)
    R = radices(n)[-1]
    NB = n // R
    for y in range(JT):
        outs = sorted(j + r * NB for j0 in range(0, NB, JT) for j in [j0 + y] for r in range(R))
        assert outs == list(range(y, n, JT))


def test_sizes_without_the_mapping_keep_the_stored_path():
    # 360 ends in radix 3 (120 butterflies per pencil, not whole rounds of 32
    # or 64 threads) and 64 in radix 8 (8 butterflies): the y-pass stores
    # their last stage and reads it back
    assert not fusable(360, 8, 256) and not fusable(360, 8, 512)
    assert not fusable(64, 8, 256) and not fusable(64, 8, 512)
