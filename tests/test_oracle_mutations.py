"""The oracle's pins catch plausible mistakes: each mutation below plants one
in a copy of ``oracle/awo_oracle.c`` (a dropped term, a flipped sign, a
transposed operand, a wrong index or tie rule -- in the particle path, the
terrain stages, the mipmap, compose, snow cover and the soft-deposit
forward and gradient), and the oracle's own pin
tests, run against the mutated copy in a sandbox, must fail.  The unmutated
copy must pass.  Nothing here touches the repository's oracle build."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor


ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
SRC = os.path.join(ROOT, "oracle", "awo_oracle.c")

PIN_FILES = ["test_oracle_closed_forms.py", "test_oracle_bruteforce.py", "test_oracle_invariants.py",
             "test_oracle_philox.py", "test_oracle_normals_release.py", "test_oracle_lod.py",
             "test_oracle_release_texture.py", "test_oracle_compose_snow.py", "test_oracle_soft.py"]

# (name, exact text in awo_oracle.c, replacement)
MUTATIONS = [
    ("bilinear weights transposed", "real top = f->h00 * ox + f->h10 * f->fx;",
     "real top = f->h00 * f->fx + f->h10 * ox;"),
    ("gradient sign", "*gx = -a * inv;", "*gx = a * inv;"),
    ("energy drop reversed", "real e1 = (e - kD * e) + (z - z1) - muD;",
     "real e1 = (e - kD * e) + (z1 - z) - muD;"),
    ("friction term dropped", "real e1 = (e - kD * e) + (z - z1) - muD;",
     "real e1 = (e - kD * e) + (z - z1);"),
    ("uniforms swapped", "real xix = uniform_pm1(wx), xiy = uniform_pm1(wy);\n\n        real rx",
     "real xix = uniform_pm1(wy), xiy = uniform_pm1(wx);\n\n        real rx"),
    ("persistence weights swapped", "\n\n        real rx = (P * dx + oneP * gx) + R * xix;",
     "\n\n        real rx = (oneP * dx + P * gx) + R * xix;"),
    ("visited-cell tie rule", "(u - (real)i0) >= (real)0.5", "(u - (real)i0) > (real)0.5"),
    ("energy tie continues", "if (!(e1 > (real)0)) { end = END_STOPPED; break; }",
     "if (!(e1 >= (real)0)) { end = END_STOPPED; break; }"),
    ("Philox counter words swapped", "uint32_t ctr[4] = {cell, j, n >> 1, 0u};",
     "uint32_t ctr[4] = {j, cell, n >> 1, 0u};"),
    ("Philox key schedule", "#define PHILOX_W0 0x9E3779B9u", "#define PHILOX_W0 0x9E3779B1u"),
    ("Philox word permutation", "uint32_t y0 = hi1 ^ x1 ^ k0;", "uint32_t y0 = hi0 ^ x1 ^ k0;"),
    ("footprint clamp dropped", "f.i1 = f.i0 + 1 < W ? f.i0 + 1 : W - 1;", "f.i1 = f.i0 < W - 1 ? f.i0 : W - 1;"),
    ("normal denominator", "real den = cs * (real)(xr - xl);", "real den = cs * (real)2;"),
    ("release bound exclusive", "int sel = (t_lo <= tan2[i]) && (tan2[i] <= t_hi);",
     "int sel = (t_lo < tan2[i]) && (tan2[i] <= t_hi);"),
    ("texel centre offset", "double c = ldexp((double)a + 0.5, -r) - 0.5;", "double c = ldexp((double)a, -r) - 0.5;"),
    ("mipmap count wraps", "sum > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)sum", "(uint32_t)sum"),
    ("colour ramp step reversed", "const real c = c0 + t * (c1 - c0);", "const real c = c1 + t * (c0 - c1);"),
    ("blend weights swapped", "to_u8(a * c + ((real)1 - a) * (real)base[4 * i + ch])",
     "to_u8(((real)1 - a) * c + a * (real)base[4 * i + ch])"),
    ("smoothstep polynomial", "return t * t * ((real)3 - (real)2 * t);", "return t * ((real)3 - (real)2 * t);"),
    ("snow slope edges swapped", "const real c0 = (real)cos(s_lo * r), c1 = (real)cos(s_hi * r);",
     "const real c0 = (real)cos(s_hi * r), c1 = (real)cos(s_lo * r);"),
    ("soft remainder dropped", "deposit[sp.cell[sp.n]] += w * sp.S[sp.n];", ";"),
    ("soft survival sign", "double S1 = S / (1.0 + exp(-e1 / tau));", "double S1 = S / (1.0 + exp(e1 / tau));"),
    ("adjoint drag factor dropped", "double lam = abar[m] * sp.S[m - 1] * dsig + (1.0 - kD) * lam_next;",
     "double lam = abar[m] * sp.S[m - 1] * dsig + lam_next;"),
]


def _sandbox(dst: str, source: str):
    os.makedirs(os.path.join(dst, "oracle"))
    for f in ("__init__.py", "build.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    with open(os.path.join(dst, "oracle", "awo_oracle.c"), "w") as f:
        f.write(source)
    os.makedirs(os.path.join(dst, "tests"))
    for f in ["__init__.py", "conftest.py", "fp64_paths.py"] + PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), os.path.join(dst, "pytest.ini"))
    os.symlink(os.path.join(ROOT, "paper_2506_23364_gb300"), os.path.join(dst, "paper_2506_23364_gb300"))


def _run(dst: str) -> int:
    env = dict(os.environ, PYTHONPATH=dst, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *[os.path.join("tests", f) for f in PIN_FILES]],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


def test_every_mutation_fails_a_pin(tmp_path):
    with open(SRC) as f:
        source = f.read()
    jobs = [("original", source)]
    for name, old, new in MUTATIONS:
        assert source.count(old) == 1, f"mutation target not found or not unique: {name}"
        jobs.append((name, source.replace(old, new, 1)))
    dirs = []
    for k, (name, text) in enumerate(jobs):
        d = os.path.join(str(tmp_path), f"m{k:02d}")
        _sandbox(d, text)
        dirs.append(d)
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        codes = list(ex.map(_run, dirs))
    assert codes[0] == 0, "the unmutated oracle copy must pass its pins"
    survivors = [name for (name, _), rc in zip(jobs[1:], codes[1:]) if rc == 0]
    assert not survivors, f"mutations no pin caught: {survivors}"
