"""Process-wide state of the library under concurrent host threads, without a
GPU: the radix-schedule cache that every context shares (kdefft_radix_plan
reads it through the same lock as the transforms' set-up).  Eight threads
request every admissible length in different orders while the cache is
being filled; each answer must equal the sequential one and be a valid
factorisation.  ctypes releases the interpreter lock during the calls, so
the threads really run inside the library at the same time."""
import math
import random
import threading

import pytest


def _smooth(x):
    for p in (2, 3, 5):
        while x % p == 0:
            x //= p
    return x == 1


def test_concurrent_radix_plan_lookups_agree():
    from paper_1511_07482_gb300 import _lib
    try:
        _lib.load()
    except RuntimeError:
        pytest.skip("libkdefft.so is not built")
    lengths = [p for p in range(2, 4097) if _smooth(p)]
    caps = [32, 16, 8]
    results = {}
    errors = []

    def worker(seed):
        rnd = random.Random(seed)
        order = [(p, c) for p in lengths for c in caps]
        rnd.shuffle(order)
        mine = {}
        try:
            for p, c in order:
                mine[(p, c)] = tuple(_lib.radix_plan(p, c))
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)
        results[seed] = mine

    threads = [threading.Thread(target=worker, args=(s,)) for s in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    ref = results[0]
    for s in range(1, 8):
        assert results[s] == ref
    for (p, c), rad in ref.items():
        assert math.prod(rad) == p and max(rad) <= c, (p, c, rad)
    # the same answers once the cache is full
    for (p, c), rad in list(ref.items())[:200]:
        assert tuple(_lib.radix_plan(p, c)) == rad
    with pytest.raises(_lib.KdefftError):
        _lib.radix_plan(7 * 16, 32)
