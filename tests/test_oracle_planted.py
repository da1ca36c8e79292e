"""Each planted mistake of the oracle must make at least one pin fail (no GPU).

The variants are the same C file compiled with -DORACLE_PLANT=k; they exist only here."""
import pytest

import oracle
import oracle_pins as P


@pytest.mark.parametrize("plant", sorted(P.PLANTS), ids=[P.PLANTS[k] for k in sorted(P.PLANTS)])
def test_planted_mistake_is_caught(plant):
    oracle.build(plant)
    failed = []
    for pin in P.PINS:
        try:
            ok, _ = pin(plant=plant)
        except Exception:  # a crash of a pin on a broken oracle also counts as caught
            ok = False
        if not ok:
            failed.append(pin.__name__)
            break
    assert failed, f"no pin caught planted mistake {plant}: {P.PLANTS[plant]}"
