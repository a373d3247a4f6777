"""Host-side checks of the candidate-ranking keys used by the GPU preselection
(Sec. 3: the H' candidates of a point are its H' largest selection scores,
ties to the lower latent index).

The kernels rank latents by a packed 32-bit key: the order-preserving key of
the FP32 score rounded down to its top 24 bits, with 255 - h in the low byte.
The FP32 form accepts the packed-key winners only when the H'-th and the
(H'+1)-th winner differ in the 24-bit prefix, and otherwise falls back to the
exact selection.  These tests restate that rule in numpy and check, on random
and adversarial (near-tied, exactly tied, many-equal) score vectors, that the
accepted sets are always the exact top-H' and that ties go to the lower h.
"""
import numpy as np
import pytest


def order_key(s):
    b = np.asarray(s, np.float32).view(np.uint32).astype(np.uint64)
    neg = (b >> 31) == 1
    return np.where(neg, (~b) & 0xFFFFFFFF, b | 0x80000000).astype(np.uint64)


def packed_keys(s):
    h = np.arange(len(s), dtype=np.uint64)
    return (order_key(s) & 0xFFFFFF00) | (255 - h)


def exact_top(s, hp):
    # descending score, ties to the lower h
    idx = sorted(range(len(s)), key=lambda h: (-float(np.float32(s[h])), h))
    return set(idx[:hp])


def packed_select(s, hp):
    pk = packed_keys(s)
    order = np.argsort(-pk.astype(np.int64), kind="stable")
    win = [int(255 - (pk[i] & 0xFF)) for i in order[:hp + 1]]
    wl, wn = pk[order[hp - 1]], pk[order[hp]] if hp < len(s) else None
    exact_ok = wn is None or (int(wl) >> 8) != (int(wn) >> 8)
    return set(win[:hp]), exact_ok


def cases(rng):
    for _ in range(300):
        yield rng.standard_normal(256).astype(np.float32)
    for _ in range(200):       # clusters of scores within a few ulps of each other
        base = rng.standard_normal(256).astype(np.float32)
        k = rng.integers(0, 256, size=40)
        base[k] = np.float32(1.5) + rng.integers(-3, 4, size=40).astype(np.float32) * np.float32(2 ** -22)
        yield base
    for _ in range(50):        # exact ties and all-equal scores
        base = np.round(rng.standard_normal(256) * 4).astype(np.float32) / 4
        yield base
    yield np.zeros(256, np.float32)
    yield -np.abs(rng.standard_normal(256)).astype(np.float32)


@pytest.mark.parametrize("hp", [1, 5, 10])
def test_accepted_packed_sets_are_exact(hp):
    rng = np.random.default_rng(1234 + hp)
    accepted = rejected = 0
    for s in cases(rng):
        got, ok = packed_select(s, hp)
        if ok:
            accepted += 1
            assert got == exact_top(s, hp)
        else:
            rejected += 1
    assert accepted > 300          # the exact fallback is the rare path
    assert rejected > 0            # and the adversarial cases do reach it


def test_packed_ties_go_to_the_lower_latent():
    s = np.zeros(256, np.float32)
    s[[7, 3, 200, 100]] = 2.0
    got, ok = packed_select(s, 2)
    assert got == {3, 7}
    assert not ok or got == exact_top(s, 2)


def test_order_key_is_monotone():
    rng = np.random.default_rng(5)
    v = np.sort(np.concatenate([rng.standard_normal(10000).astype(np.float32),
                                np.array([-np.inf, 0.0, np.inf], np.float32)]))
    k = order_key(v)
    assert np.all(np.diff(k.astype(np.int64)) >= 0)
