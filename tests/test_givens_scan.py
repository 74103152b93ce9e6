"""The Givens update of a new Hessenberg column as a scan of affine maps.

Least squares in GMRES (Section 5) applies the j stored rotations (c_i, s_i) to each
new column h.  The sequential loop carries one running entry a_i (a_0 = h_0):

  out_i   = c_i a_i + s_i h_{i+1}
  a_{i+1} = -conj(s_i) a_i + c_i h_{i+1}

The second line makes a_{i+1} an affine function of a_i, a -> m_i a + t_i with
m_i = -conj(s_i) and t_i = c_i h_{i+1}.  So the chain of a's is a prefix composition
of affine maps.  The GPU's Givens kernel works this way: each lane composes the
maps of one segment, a Kogge-Stone scan over the segments gives every segment its
incoming value, and each segment is then replayed from that value.  This takes
2 j / S + log2 S dependent steps instead of j.

Here the formulation is restated in NumPy (segments, inclusive scan by doubling,
replay) and checked against the sequential loop.  Since |m_i| <= 1, the composed
maps stay bounded and the two agree to rounding for columns of up to 1000 rotations.
"""
import numpy as np
import pytest

from oracle import givens


def sequential(cs, sn, h):
    a = h[0]
    out = np.empty(len(cs), dtype=np.complex128)
    for i in range(len(cs)):
        out[i] = cs[i] * a + sn[i] * h[i + 1]
        a = -np.conj(sn[i]) * a + cs[i] * h[i + 1]
    return out, a


def compose(f, g):
    """g after f for affine maps (m, t): x -> m x + t."""
    return g[0] * f[0], g[0] * f[1] + g[1]


def scan_form(cs, sn, h, segments):
    j = len(cs)
    m = -np.conj(sn)
    t = cs * h[1:j + 1]
    bounds = np.linspace(0, j, segments + 1).astype(int)
    seg = []
    for k in range(segments):                       # each lane composes its segment's maps
        acc = (1.0 + 0j, 0j)
        for i in range(bounds[k], bounds[k + 1]):
            acc = compose(acc, (m[i], t[i]))
        seg.append(acc)
    incl = list(seg)                                # inclusive scan by doubling (Kogge-Stone)
    d = 1
    while d < segments:
        incl = [compose(incl[k - d], incl[k]) if k >= d else incl[k] for k in range(segments)]
        d *= 2
    out = np.empty(j, dtype=np.complex128)
    for k in range(segments):                       # replay each segment from its incoming value
        a = h[0] if k == 0 else incl[k - 1][0] * h[0] + incl[k - 1][1]
        for i in range(bounds[k], bounds[k + 1]):
            out[i] = cs[i] * a + sn[i] * h[i + 1]
            a = m[i] * a + t[i]
    total = incl[-1]
    return out, total[0] * h[0] + total[1]


@pytest.mark.parametrize("j", [1, 2, 7, 127, 128, 129, 513, 1000])
@pytest.mark.parametrize("segments", [4, 128])
def test_scan_form_equals_sequential_rotations(j, segments):
    rng = np.random.default_rng(j * 7 + segments)
    cs = np.empty(j)
    sn = np.empty(j, dtype=np.complex128)
    for i in range(j):                              # rotations as GMRES forms them
        a, b = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        cs[i], sn[i] = givens(a, b)
    h = rng.standard_normal(j + 1) + 1j * rng.standard_normal(j + 1)
    out_s, a_s = sequential(cs, sn, h)
    out_k, a_k = scan_form(cs, sn, h, min(segments, j))
    scale = np.linalg.norm(h)
    assert np.max(np.abs(out_k - out_s)) <= 1e-13 * scale
    assert abs(a_k - a_s) <= 1e-13 * scale
    # the rotations are unitary: the column keeps its 2-norm
    assert np.sqrt(np.sum(np.abs(out_s) ** 2) + abs(a_s) ** 2) == pytest.approx(scale, rel=1e-12)
