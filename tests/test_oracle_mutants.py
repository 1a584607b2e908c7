"""Planted mistakes in the oracle (CPU only): each mutant copy of the oracle
source must fail at least one pin, which shows the pins would catch that
class of error (a dropped term, a wrong sign or index, a transposed operand)."""
import numpy as np
import pytest

import oracle
from tests import oracle_pins as P

MUTANTS = {
    "rx_sign": ("m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c;",
                "m[0] = c; m[1] = I * s; m[2] = I * s; m[3] = c;"),
    "ry_transposed": ("m[0] = c; m[1] = -s; m[2] = s; m[3] = c;",
                      "m[0] = c; m[1] = s; m[2] = -s; m[3] = c;"),
    "rz_half_angle_dropped": ("m[3] = cexp(0.5 * I * p[0]);", "m[3] = cexp(I * p[0]);"),
    "u3_phi_lambda_swapped": ("m[1] = -cexp(I * p[2]) * s;", "m[1] = -cexp(I * p[1]) * s;"),
    "cx_control_target_swapped": ("m[0 * 4 + 0] = 1; m[1 * 4 + 1] = 1; m[2 * 4 + 3] = 1; m[3 * 4 + 2] = 1;",
                                  "m[0 * 4 + 0] = 1; m[2 * 4 + 2] = 1; m[1 * 4 + 3] = 1; m[3 * 4 + 1] = 1;"),
    "local_bit_order": ("if ((j >> (k - 1 - i)) & 1) o |= 1ull << q[i];",
                        "if ((j >> i) & 1) o |= 1ull << q[i];"),
    "matvec_transposed": ("acc += m[a * d + b] * v[b];", "acc += m[b * d + a] * v[b];"),
    "sampler_ge": ("if (c[mid] > t) hi = mid;", "if (c[mid] >= t) hi = mid;"),
    "expect_z_sign": ("ez[i] += ((x >> i) & 1) ? -p : p;", "ez[i] += ((x >> i) & 1) ? p : -p;"),
    "probs_dropped_imag": ("p[x] = psi_ri[2 * x] * psi_ri[2 * x] + psi_ri[2 * x + 1] * psi_ri[2 * x + 1];",
                           "p[x] = psi_ri[2 * x] * psi_ri[2 * x];"),
    "philox_wrong_word": ("uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;",
                          "uint64_t n0 = hi0 ^ c1 ^ k0, n1 = lo1, n2 = hi1 ^ c3 ^ k1, n3 = lo0;"),
    "cp_phase_on_wrong_entry": ("m[15] = (type == G_CZ) ? -1.0 : cexp(I * p[0]);",
                                "m[15] = (type == G_CZ) ? -1.0 : cexp(-I * p[0]);"),
}


def _fails_some_pin(O):
    checks = P.ALL_STATE_CHECKS
    for chk in checks:
        try:
            chk(O, np.random.default_rng(3))
        except AssertionError:
            return chk.__name__
        except StopIteration:
            return chk.__name__
    return None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, name
    O = oracle.compile_variant(src.replace(old, new), str(tmp_path / ("m_" + name + ".so")))
    caught = _fails_some_pin(O)
    assert caught is not None, "mutant %s passed every pin" % name
