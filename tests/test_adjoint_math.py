"""The hand-written reverse-mode derivative of the contact law (dem_contact.cuh)
against fourth-order central differences of the same law, both compiled for the
host in double precision (CPU only)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_contact_vjp_matches_finite_differences(tmp_path):
    exe = tmp_path / "vjp"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                           os.path.join(ROOT, "paper_1705_03850_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "contact_vjp_check.cpp"), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    res = {l.split()[0]: (float(l.split()[1]), int(l.split()[2])) for l in out if l.strip()}
    # slip cases exercise the Coulomb branch, stick cases mostly the spring branch
    assert res["pair_slip"][1] == 200 and res["wall_slip"][1] == 200
    assert res["pair_stick"][1] < 200 and res["wall_stick"][1] < 200
    assert res["pair_stick"][0] < 1e-5 and res["wall_stick"][0] < 1e-5
    assert res["pair_slip"][0] < 1e-3 and res["wall_slip"][0] < 1e-3
