"""Planted mistakes: the oracle is rebuilt with one plausible mistake at a time (a dropped
flux term, a flipped sign, a wrong neighbour row, an unlimited flux, a wrong time
weight, a fixed axis order, ...; see ORC_MUTANT in oracle/mhd_oracle.c) and at least one
pin must fail for each.  This shows the pins are sharp enough to catch such mistakes in
the oracle itself.  CPU only; mistakes are planted in the oracle, never in the CUDA path."""
import pytest

import oracle
import pins

# mutant id -> the pins expected to catch it (a subset of what does; kept cheap)
MUTANTS = {
    1: ("dropped -B_n B_t1 in the transverse momentum flux", ["alfven"]),
    2: ("flipped sign of the advection update of B_t", ["divb_ot", "entropy_wave"]),
    3: ("constraint uses the row below instead of above", ["conservation", "divb_ot"]),
    4: ("unlimited (central) second-order correction", ["tvd_contact", "limiter"]),
    5: ("wrong sign of the left-moving correction", ["entropy_wave", "sod"]),
    6: ("face velocity divides by the density on the wrong side", ["passive_field"]),
    7: ("magnetic pressure dropped from the equation of state", ["fast_wave"]),
    8: ("freezing speed without the magnetic term", ["alfven", "embedding"]),
    9: ("no cycling of the axis order", ["phase_cycling", "permutation"]),
    10: ("reverse sweep not reversed", ["fast_wave"]),
    11: ("time step not scaled by the cell width", ["entropy_wave", "sod"]),
    12: ("a step advances dt instead of 2 dt", ["entropy_wave", "sod"]),
    13: ("predictor over a full dt", ["entropy_wave", "sod"]),
    14: ("(1,2,1) smoothing summed from one side", ["mirror"]),
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant):
    what, names = MUTANTS[mutant]
    oracle.build(mutant)
    failed = []
    for name in names:
        ok, detail = pins.ALL_PINS[name](mutant=mutant)
        if not ok:
            failed.append(f"{name}: {detail}")
    assert failed, f"mutant {mutant} ({what}) passed the pins {names}"


def test_default_build_has_no_mutant():
    assert oracle.load(0).orc_mutant() == 0
