"""Pins of the oracle's padding geometry (Sec. III.B, Eq. (1)-(2)) and of the
symmetric padding (Algorithm 1, first two steps) against hand values, brute
force and numpy's own symmetric padding."""
import numpy as np
import pytest

# (s, b) -> (p, p0, p1, n), worked by hand from Eq. (1)-(2)
HAND = {
    (512, 64): (64, 32, 32, 9),
    (32, 8): (8, 4, 4, 5),
    (64, 16): (16, 8, 8, 5),
    (4, 2): (2, 1, 1, 3),
    (5, 2): (3, 1, 2, 4),
    (4, 3): (5, 2, 3, 3),
    (1, 1): (1, 0, 1, 2),
    (7, 7): (7, 3, 4, 2),
}


@pytest.mark.parametrize("sb", sorted(HAND))
def test_padding_hand_values(orc, sb):
    s, b = sb
    g = orc.geometry([s], [b])
    assert (g["p"][0], g["p0"][0], g["p1"][0], g["n"][0]) == HAND[sb]


def test_padding_brute_force(orc):
    # Sec. III.B: pad to a multiple of b, then by b more; so p is the unique
    # value in [b, 2b-1] with (s + p) divisible by b.  Every voxel must then
    # lie between the first and the last kernel centre k*b + (b-1)/2.
    for s in range(1, 41):
        for b in range(1, s + 1):
            g = orc.geometry([s], [b])
            p, p0, p1, n = g["p"][0], g["p0"][0], g["p1"][0], g["n"][0]
            want = [q for q in range(b, 2 * b) if (s + q) % b == 0]
            assert want == [p]
            assert p0 + p1 == p and p0 == p // 2
            assert n * b == s + p
            centres = [k * b + (b - 1) / 2 for k in range(n)]
            for x in range(s):
                P = x + p0
                assert centres[0] <= P < centres[-1]


def test_geometry_rejects_kernel_larger_than_volume(orc):
    with pytest.raises(ValueError):
        orc.geometry([4], [5])
    with pytest.raises(ValueError):
        orc.geometry([4, 4], [2, 0])


@pytest.mark.parametrize("ndim", [1, 2, 3, 4])
def test_symmetric_padding_matches_numpy(orc, ndim):
    rng = np.random.default_rng(10 + ndim)
    for _ in range(6):
        shape = tuple(int(v) for v in rng.integers(1, 9 if ndim < 4 else 6, size=ndim))
        ks = tuple(int(rng.integers(1, s + 1)) for s in shape)
        x = rng.random(shape, dtype=np.float32)
        g = orc.geometry(shape, ks)
        want = np.pad(x, list(zip(g["p0"], g["p1"])), mode="symmetric")
        np.testing.assert_array_equal(orc.pad(x, ks), want)
