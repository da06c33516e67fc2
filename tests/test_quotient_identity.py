"""The integration's update divides by W + 1 (an integer 1..256 with the
constant weight) and by mu.  The planned replacement of those two IEEE
divisions, the quotient from a correctly rounded reciprocal corrected by two
fused multiply-adds (Markstein 1990), must return the IEEE quotient itself.
This CPU test checks that exhaustively over the float significands of the
numerator for every such divisor, the mu of every configuration and batched
scene, and 200 pseudo-random divisors (for the projection's quotients by a
voxel's depth, which could share one reciprocal); the same
IEEE operations round identically on the GPU.  As a control, the uncorrected
product a * RN(1/d) must differ from the quotient somewhere."""

import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_corrected_reciprocal_quotient_is_the_ieee_quotient(tmp_path):
    exe = str(tmp_path / "quotient_check")
    try:
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-o", exe,
                               os.path.join(HERE, "quotient_check.c"), "-lm"])
    except (OSError, subprocess.CalledProcessError) as e:  # pragma: no cover - no OpenMP compiler
        pytest.skip("cannot build the check: %s" % e)
    from synth import batched, workload_by_name
    mus = {workload_by_name(n, n_frames=2).params["mu"] for n in ("tiny", "kinect", "large")}
    mus |= {w.params["mu"] for w in batched.small_scenes()} | {0.032}
    mus = ["%.9g" % m for m in sorted(mus)]
    out = subprocess.run([exe, "200", *mus], capture_output=True, text=True, timeout=600,
                         check=True).stdout.split()
    bad, bad_q0 = int(out[0]), int(out[1])
    assert bad == 0
    assert bad_q0 > 10 ** 8
