"""The oracle's pins reject plausible mistakes.

Each case plants one mistake in a copy of the oracle (a dropped term, a
wrong sign, a transposed operand, a wrong constant or factor), builds the copy
in a scratch directory and runs the pin suites (tests/test_oracle_pins.py,
tests/test_oracle_dy.py) against it in a subprocess; at least one pin must fail.  The unmodified copy
must pass, so a failure is the mistake's doing.  CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, exact source text, replacement): one occurrence each
MUTATIONS = [
    ("three-gluon vertex drops a term",
     "out[mu] = j12 * d12[mu] + J2[mu] * a + J1[mu] * b;", "out[mu] = j12 * d12[mu] + J2[mu] * a;"),
    ("slash: sign of a spatial component",
     "- GAM[1][r][c] * J[1] - GAM[2][r][c] * J[2]", "+ GAM[1][r][c] * J[1] - GAM[2][r][c] * J[2]"),
    ("row-vector product transposed", "for (int r = 0; r < 4; ++r) s += x[r] * M[r][c];",
     "for (int r = 0; r < 4; ++r) s += x[r] * M[c][r];"),
    ("quark propagator: sign of the mass term",
     "            double den = mdot(q, q) - mt * mt;\n            for (int c = 0; c < 4; ++c) U[j][c]",
     "            double den = mdot(q, q) + mt * mt;\n            for (int c = 0; c < 4; ++c) U[j][c]"),
    ("four-gluon vertex coefficient", "tmp[mu] += I * (2.0 * ac * B[mu] - ab * Cc[mu] - bc * A[mu]);",
     "tmp[mu] += I * (1.0 * ac * B[mu] - ab * Cc[mu] - bc * A[mu]);"),
    ("polarisation vector: sign of the imaginary part", "(-lam * e1[mu] - I * e2[mu]) / sqrt(2.0)",
     "(-lam * e1[mu] + I * e2[mu]) / sqrt(2.0)"),
    ("spinor: small component without the square root", "*wm = (m == 0.0) ? 0.0 : sqrt(m * m / (E + P));",
     "*wm = (m == 0.0) ? 0.0 : m * m / (E + P);"),
    ("two-spinor: wrong phase", "else { out[0] = (-px + I * py) / n; out[1] = ppz / n; }",
     "else { out[0] = (px + I * py) / n; out[1] = ppz / n; }"),
    ("Philox multiplier constant", "PHILOX_M0 = 0xD2E7470EE14C6C93ULL", "PHILOX_M0 = 0xD2E7470EE14C6C95ULL"),
    ("uniform offset", "((double)(x >> 11) + 0.5) * 0x1p-53", "((double)(x >> 11) + 1.0) * 0x1p-53"),
    ("RAMBO boost: missing term", "mom[j][i + 1] = x * (q[j][i + 1] + b[i] * q[j][0] + a * bq * b[i]);",
     "mom[j][i + 1] = x * (q[j][i + 1] + b[i] * q[j][0]);"),
    ("SU(3) generator sign", "TG[1][0][1] = -0.5 * I; TG[1][1][0] = 0.5 * I;",
     "TG[1][0][1] = 0.5 * I; TG[1][1][0] = 0.5 * I;"),
    ("identical-gluon factor", "return 4.0 * 64.0 * factorial(proc - 1);", "return 4.0 * 64.0 * factorial(proc);"),
    ("Drell-Yan: Z right-handed coupling sign", "*gr = -e * q * sw * sw / (sw * cw);",
     "*gr = e * q * sw * sw / (sw * cw);"),
    ("Drell-Yan: quark chiralities swapped at the insertion", "M[r][c] += S[r][c] * (c < 2 ? gl : gr);",
     "M[r][c] += S[r][c] * (c < 2 ? gr : gl);"),
    ("Drell-Yan: insertion propagator misses the lepton-pair momentum",
     "for (int mu = 0; mu < 4; ++mu) q1[mu] = q0[mu] + qL[mu];", "for (int mu = 0; mu < 4; ++mu) q1[mu] = q0[mu];"),
    ("diagram weights: four-gluon structure repeated",
     "cur[t][v + 1][mu] = inv * (ab * C[mu] - bc * A[mu]);", "cur[t][v + 1][mu] = inv * (ab * C[mu] - ac * B[mu]);"),
    ("diagram weights: three-gluon vertex legs' momenta swapped",
     "v3(cur[a][va], ka, cur[b][vb], kb, o);", "v3(cur[a][va], kb, cur[b][vb], ka, o);"),
    ("diagram weights: sign of the top mass in the propagator denominator",
     "const double den = mdot(q, q) - mt * mt;", "const double den = mdot(q, q) + mt * mt;"),
]

# the heaviest pins are not needed to catch these mistakes
PIN_SELECTION = "not k5 and not some_helicities and not ttxggg"


def run_pins(workdir):
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
           os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_dy.py"),
           "-k", PIN_SELECTION]
    r = subprocess.run(cmd, cwd=workdir, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def oracle_copy(tmp_path, mutation=None):
    work = tmp_path / "w"
    pkg = work / "oracle"
    pkg.mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg / "__init__.py")
    src = open(os.path.join(ROOT, "oracle", "me_oracle.c")).read()
    if mutation:
        _, old, new = mutation
        assert src.count(old) == 1, mutation[0]
        src = src.replace(old, new)
    (pkg / "me_oracle.c").write_text(src)
    return work


@pytest.mark.slow
def test_unmodified_copy_passes(tmp_path):
    rc, out = run_pins(oracle_copy(tmp_path))
    assert rc == 0, out


@pytest.mark.slow
@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_reject_mutation(tmp_path, mutation):
    rc, out = run_pins(oracle_copy(tmp_path, mutation))
    assert rc != 0, f"{mutation[0]}: no pin failed\n{out}"
