"""The FastILU pins of tests/test_oracle_ilu.py as one function returning
the names of those that fail, for the mutation test."""
import numpy as np

import gen
import test_oracle_ilu as t


def failures(orc):
    bad = set()

    def check(name, fn):
        try:
            fn()
        except Exception:
            bad.add(name)

    check("levels", lambda: t.test_iluk_pattern_brute_force(orc, 2, 2))
    check("complete fill", lambda: t.test_complete_fill_is_exact_lu(orc, "random"))
    check("hand sweeps", lambda: t.test_first_sweeps_by_hand(orc))
    check("fixed point", lambda: t.test_exact_factors_are_the_fixed_point(orc, 1))
    check("trsv lower", lambda: t.test_fast_trsv_exact_after_n_sweeps(orc, 0))
    check("trsv upper", lambda: t.test_fast_trsv_exact_after_n_sweeps(orc, 1))
    return bad
