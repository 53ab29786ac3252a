"""Pin sensitivity: plausible mistakes planted in a temporary copy of the oracle must each make
at least one pin fail.

Each mutation is a text substitution applied to a copy of oracle.c in a temporary folder and
built there on the CPU; the committed oracle carries no trace of them.  Every original snippet
must occur exactly once in oracle.c, so a mutation cannot silently stop applying when the
oracle is edited.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# k: (what the mistake is, original text, mistaken text)
MUTATIONS = {
    1: ("drops cos(elevation) from the channel phase",
        "o->nu_a = spacing_wl(p) * sin(az) * cos(el);",
        "o->nu_a = spacing_wl(p) * sin(az);"),
    2: ("flips the sign of the Doppler term",
        "o->nu_d = p->carrier_hz * (2.0 * v * p->chirp_period_s) / ORC_C;",
        "o->nu_d = -(p->carrier_hz * (2.0 * v * p->chirp_period_s) / ORC_C);"),
    3: ("uses the sweep time T_c as the chirp period",
        "o->nu_d = p->carrier_hz * (2.0 * v * p->chirp_period_s) / ORC_C;",
        "o->nu_d = p->carrier_hz * (2.0 * v * p->sweep_time_s) / ORC_C;"),
    4: ("treats the path length as one-way in the beat frequency",
        "o->nu_r = mu * dt * tau;",
        "o->nu_r = mu * dt * tau / 2.0;"),
    5: ("drops the start phase phi0",
        "o->carrier = frac(p->carrier_hz * tau) + frac((double)r->phase0_rad[i] / ORC_TWO_PI);",
        "o->carrier = frac(p->carrier_hz * tau);"),
    6: ("truncates instead of rounding bin coordinates",
        "int64_t q = (int64_t)floor(x + 0.5);",
        "int64_t q = (int64_t)floor(x);"),
    7: ("breaks label ties toward the largest id",
        "if (e[t] > best_e) {",
        "if (e[t] >= best_e) {"),
    8: ("leaves the range window out of the spectrum",
        "dft_ctx c0 = {p, signal, t1, wr, tr, 0};",
        "for (int64_t t = 0; t < ns; ++t) wr[t] = 1.0;\n  dft_ctx c0 = {p, signal, t1, wr, tr, 0};"),
    9: ("uses sin(elevation) in the antenna pattern",
        "const double c = orc_cos_rep(az) * orc_cos_rep(el);",
        "const double c = orc_cos_rep(az) * orc_sin_rep(el);"),
    10: ("takes the receiver index as the TDM transmitter slot",
         "return k / p->n_rx;",
         "return k % p->n_rx;"),
    11: ("swaps the barycentric weights u and v of Eq. 6",
         "out[c] = w * V[3 * tri[0] + c] + u * V[3 * tri[1] + c] + v * V[3 * tri[2] + c];",
         "out[c] = w * V[3 * tri[0] + c] + v * V[3 * tri[1] + c] + u * V[3 * tri[2] + c];"),
    12: ("measures the receiver leg of Eq. 7 to the transmitter's position",
         "distance3(plj, g->rx_pos + 3 * rx);",
         "distance3(plj, g->rx_pos + 3 * t);"),
}


def test_every_mutation_applies_once():
    src = open(SRC).read()
    for k, (what, orig, _) in MUTATIONS.items():
        assert src.count(orig) == 1, f"mutation {k} ({what}): original text found {src.count(orig)} times"
    assert "MUTATION" not in src


@pytest.mark.parametrize("k", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(k, tmp_path):
    what, orig, bad = MUTATIONS[k]
    src = open(SRC).read()
    assert src.count(orig) == 1
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(src.replace(orig, bad))
    for h in ("oracle.h",):
        (tmp_path / h).write_text(open(os.path.join(ROOT, "oracle", h)).read())
    lib = tmp_path / f"liboracle_mut{k}.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                           "-o", str(lib), str(mutant), "-lm", "-lpthread"])
    env = dict(os.environ, RADAR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")], env=env, capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"no pin caught mutation {k} ({what})"
    assert "failed" in r.stdout
