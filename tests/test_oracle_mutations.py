"""Pin sensitivity: plausible mistakes planted in the oracle (compile-time switches of
oracle.c, built here on the CPU) must each make at least one pin fail."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    1: "drops cos(elevation) from the channel phase",
    2: "flips the sign of the Doppler term",
    3: "uses the sweep time T_c as the chirp period",
    4: "treats the path length as one-way in the beat frequency",
    5: "drops the start phase phi0",
    6: "truncates instead of rounding bin coordinates",
    7: "breaks label ties toward the largest id",
    8: "leaves the range window out of the spectrum",
    9: "uses sin(elevation) in the antenna pattern",
    10: "takes the receiver index as the TDM transmitter slot",
    11: "swaps the barycentric weights u and v of Eq. 6",
    12: "measures the receiver leg of Eq. 7 to the transmitter's position",
}


@pytest.mark.parametrize("k", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(k, tmp_path):
    lib = tmp_path / f"liboracle_mut{k}.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
                           f"-DORC_MUTATION={k}", "-o", str(lib), SRC, "-lm", "-lpthread"])
    env = dict(os.environ, RADAR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")], env=env, capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"no pin caught mutation {k} ({MUTATIONS[k]})"
    assert "failed" in r.stdout
