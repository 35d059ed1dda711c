"""The oracle's pins have teeth: each mutant below is the oracle's C source
with one plausible mistake -- a dropped term, a wrong sign, index, bound or
scale, a wrong rounding rule, a transposed operand -- and every one of them
must fail at least one pin of test_oracle*.py.  The oracle is not changed:
each mistake is a text substitution on a copy in a temporary directory,
compiled with the oracle's own flags, and the pins run against it in a child
process (a mutant that crashes counts as caught)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "emu_oracle.c")

# (name, text in the oracle, replacement, occurrence): occurrence None = the
# text must occur once; an index picks one of several identical sites
MUTANTS = [
    # Eq. 1 scale vectors: floor(log2 max) instead of the frexp exponent
    ("row exponent one low", "if (mx != 0.0) frexp(mx, &e);", "if (mx != 0.0) { frexp(mx, &e); e -= 1; }", None),
    # Scheme I split (R1)
    ("slice scale without the sign bit", "scaled_trunc(X[i * k + h], 8 * p - 1 - E[i])",
     "scaled_trunc(X[i * k + h], 8 * p - E[i])", None),
    ("wrong slice signed", "if (t == 0 && byte >= 128) byte -= 256;", "if (t == 1 && byte >= 128) byte -= 256;", None),
    ("truncation rounds", "mag = (u128)(M >> (-sh));", "mag = (u128)((M + ((uint64_t)1 << (-sh - 1))) >> (-sh));", None),
    # Eq. 11 layout
    ("slice-major interleave", "Ahat[i * nck * p * tk + (c * p + t) * tk + r]",
     "Ahat[i * nck * p * tk + (t * nck + c) * tk + r]", None),
    # chunk length of R2
    ("K_c bound one tail term too many", "(int64_t)(p - 2) * 255 * 255", "(int64_t)(p - 1) * 255 * 255", None),
    # Eq. 2 triangle / Eq. 3 shift-reduce
    ("partials drop the diagonal term", "int64_t acc = 0;\n          for (int t = 0; t <= s; ++t) {",
     "int64_t acc = 0;\n          for (int t = 0; t < s; ++t) {", None),
    # the INT8 product (orc_emu_I) comes before the E4M3 one, whose loop is the same text
    ("Scheme I pairs slice t with t", "const int16_t *b = DB + ((int64_t)(s - t) * n + j) * k;\n          for (int64_t h = 0; h < k; ++h) Cs",
     "const int16_t *b = DB + ((int64_t)t * n + j) * k;\n          for (int64_t h = 0; h < k; ++h) Cs", 0),
    ("shift-reduce weight off by one slice", "S += (i128)Cs << (8 * (p - 1 - s));", "S += (i128)Cs << (8 * (p - s));", None),
    ("Scheme I scale exponent", "E[i] + F[j] - 14 - 8 * (p - 1)", "E[i] + F[j] - 16 - 8 * (p - 1)", None),
    ("rounding ties away from zero", "if (rest > half || (rest == half && (top & 1))) top += 1;",
     "if (rest >= half) top += 1;", None),
    ("BLAS update rounds twice", "return fma(alpha, r, beta * c);", "return alpha * r + beta * c;", None),
    # Scheme II (R3, R4, Eqs. 5-8)
    ("moduli start at 255", "for (int x = 256; x >= 2 && cnt < nm; --x)", "for (int x = 255; x >= 2 && cnt < nm; --x)", None),
    ("scale bits one too many", "int num = orc_log2P_floor(nm) - (is_complex ? 2 : 1) - c;",
     "int num = orc_log2P_floor(nm) - (is_complex ? 2 : 1) - c + 1;", None),
    # (r > m / 2 would be an equivalent mutant: it differs only at r = 128
    # for m = 256, which the int8 store wraps to -128 anyway)
    ("residue range off by one", "if (r > (m - 1) / 2) r -= m;", "if (r >= (m - 1) / 2) r -= m;", None),
    ("negative remainder not lifted", "  int r = (int)(x % m);\n  if (r < 0) r += m;", "  int r = (int)(x % m);", None),
    ("output residue left negative", "        int64_t r = acc % mods[l];\n        if (r < 0) r += mods[l];",
     "        int64_t r = acc % mods[l];", None),
    ("CRT weight without the inverse", "big_mul_u32(&w, &Pl, (uint32_t)q);", "big_mul_u32(&w, &Pl, 1u);", None),
    ("CRT lift maps P/2 to -P/2", "if (big_cmp(&S, &cx->halfP_floor) > 0) {", "if (big_cmp(&S, &cx->halfP_floor) >= 0) {", None),
    ("Scheme II scale back", "double r = ldexp(v, E[i] + F[j] - bA - bB);", "double r = ldexp(v, E[i] + F[j] - bA - bB + 1);", None),
    # 3M (Eq. 16)
    ("3M real part adds T2", "int64_t re = ((t[0] - t[1]) % ml + ml) % ml;", "int64_t re = ((t[0] + t[1]) % ml + ml) % ml;", None),
    ("3M imaginary part adds T2", "int64_t im = ((t[2] - t[0] - t[1]) % ml + 2 * ml) % ml;",
     "int64_t im = ((t[2] - t[0] + t[1]) % ml + 2 * ml) % ml;", None),
    ("3M sum residue is a difference", "v = part == 0 ? re : part == 1 ? im : re + im;",
     "v = part == 0 ? re : part == 1 ? im : re - im;", None),
    ("complex alpha sign", "double tr = fma(ar, rr, -(ai * ri));", "double tr = fma(ar, rr, ai * ri);", None),
    # E4M3 slices (R7)
    ("E4M3 digit range [-15, 16]", "if (r >= 16) r -= 32;", "if (r > 16) r -= 32;", None),
    ("E4M3 scale exponent", "E[i] + F[j] - 8 - 5 * (p - 1)", "E[i] + F[j] - 10 - 5 * (p - 1)", None),
    # 4M Scheme I complex (R8)
    ("4M real part without -Im B", "tri_sum(DAi, i, m, DBn, j, n, k, s)", "tri_sum(DAi, i, m, DBi, j, n, k, s)", None),
    # norm scaling (R9)
    ("norm exponent rounds down", "int ep = d >= 0 ? (d + 1) / 2 : -((-d) / 2);",
     "int ep = d >= 0 ? d / 2 : -((-d) / 2);", None),
    ("norm halves one too many", "*hA = L >= 0 ? L / 2 : -((-L + 1) / 2);", "*hA = L >= 0 ? L / 2 + 1 : -((-L + 1) / 2);", None),
    # double-double reference
    ("dd ZGEMM real part adds Im*Im", "dot2(a, 1, b, 1, 2 * k, 1.0,", "dot2(a, 1, b, 1, 2 * k, 0.0,", None),
    ("dd dot drops the TwoSum error", "    c += err + e;\n  }\n  double t = s + c;", "    c += e;\n  }\n  double t = s + c;", None),
    ("dd ZGEMM imaginary part drops the TwoSum error", "          c += err + e;\n        }\n      }",
     "          c += e;\n        }\n      }", None),
    ("dd ZGEMM imaginary part drops the product error", "          c += err + e;\n        }\n      }",
     "          c += err;\n        }\n      }", None),
    # more of the integer and rounding machinery
    ("CRT rounding ignores the sticky bits", "if (guard && (sticky || (top & 1))) top += 1;",
     "if (guard && (top & 1)) top += 1;", None),
    ("CRT sum not reduced mod P", "    if (big_cmp(&S, &cx->P) >= 0) big_sub(&S, &S, &cx->P);\n  }\n  if (big_cmp(&S, &cx->halfP_floor) > 0)",
     "  }\n  if (big_cmp(&S, &cx->halfP_floor) > 0)", None),
    ("norm squares rounded down", "  if ((q << (-s)) != M2) q += 1;\n  return q;", "  return q;", None),
    ("E4M3 leading digit dropped", "      D[i * k + h] = (int16_t)x;", "      D[i * k + h] = 0;", None),
    ("interleave pads with ones", "int v = h < k ? D[((int64_t)t * rows + i) * k + h] : 0;",
     "int v = h < k ? D[((int64_t)t * rows + i) * k + h] : 1;", None),
    ("K_c not a multiple of 256", "  int64_t lim = 2147483647LL / bnd;\n  return (lim / 256) * 256;",
     "  int64_t lim = 2147483647LL / bnd;\n  return lim;", None),
    ("4M E4M3 scale exponent", "const int escale = f8 ? -8 - 5 * (p - 1) : -14 - 8 * (p - 1);",
     "const int escale = f8 ? -8 - 5 * p : -14 - 8 * (p - 1);", None),
    ("scaled integer loses its sign", "return a < 0 ? -(i128)mag : (i128)mag;", "return (i128)mag;", None),
    ("complex row exponent over half the row", "  return orc_row_exponents(rows, 2 * cols, X, E);",
     "  return orc_row_exponents(rows, cols, X, E);", None),
    ("multi-word subtraction borrow", "    br = d < 0;", "    br = d <= 0;", None),
    ("complex beta term subtracted", "    tr = tr + ur;", "    tr = tr - ur;", None),
    ("complex norm over the real parts only",
     "    for (int64_t h = 0; h < cols * cw; ++h) S += sq_ceil64(X[i * cols * cw + h], Emax);",
     "    for (int64_t h = 0; h < cols * cw; h += cw) S += sq_ceil64(X[i * cols * cw + h], Emax);", None),
    ("residue product skips the last K term",
     "        for (int64_t h = 0; h < k; ++h) acc += (int64_t)a[h] * (int64_t)b[h];\n        int64_t r = acc % mods[l];",
     "        for (int64_t h = 0; h + 1 < k; ++h) acc += (int64_t)a[h] * (int64_t)b[h];\n        int64_t r = acc % mods[l];",
     None),
]

# The child: load the oracle module against the mutant library and run every
# pin until one fails (exit 1) or all pass (exit 0).
RUNNER = r"""
import importlib.util, inspect, itertools, os, sys, tempfile, pathlib
root, lib, src = sys.argv[1:4]
wrapper = sys.argv[4] if len(sys.argv) > 4 else os.path.join(root, "oracle", "__init__.py")
sys.path[:0] = [root, os.path.join(root, "tests")]
import pytest
spec = importlib.util.spec_from_file_location("oracle_mutant", wrapper)
orc = importlib.util.module_from_spec(spec)
spec.loader.exec_module(orc)
orc._LIB_PATH, orc._SRC, orc._OUT_DIR = lib, src, os.path.dirname(lib)

def cases(fn):
    grids = []
    for m in getattr(fn, "pytestmark", []):
        if m.name == "skip" or (m.name == "skipif" and m.args and m.args[0]):
            return
        if m.name != "parametrize":
            continue
        names = m.args[0]
        names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
        vals = []
        for v in m.args[1]:
            if hasattr(v, "values") and hasattr(v, "marks"):
                v = v.values if len(names) > 1 else v.values[0]
            vals.append(dict(zip(names, v)) if len(names) > 1 else {names[0]: v})
        grids.append(vals)
    for combo in itertools.product(*grids):
        kw = {}
        for d in combo:
            kw.update(d)
        yield kw

for modname in ("test_oracle", "test_oracle_f8", "test_oracle_norm", "test_oracle_z4m"):
    mod = importlib.import_module(modname)
    for name, fn in sorted(vars(mod).items()):
        if not (name.startswith("test_") and callable(fn)):
            continue
        params = inspect.signature(fn).parameters
        for kw in cases(fn):
            args = {}
            for p in params:
                if p == "orc":
                    args[p] = orc
                elif p == "tmp_path":
                    args[p] = pathlib.Path(tempfile.mkdtemp())
                elif p in kw:
                    args[p] = kw[p]
                else:
                    args = None
                    break
            if args is None:
                continue
            try:
                fn(**args)
            except pytest.skip.Exception:
                continue
            except Exception as e:
                print("caught by", modname + "::" + name, kw, type(e).__name__)
                sys.exit(1)
print("survived every pin")
sys.exit(0)
"""


def mutate(text, old, new, which):
    """Replace occurrence `which` (None: the only one) of `old` by `new`."""
    pos = -1
    for _ in range((which or 0) + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, f"mutation site not found: {old!r}"
    return text[:pos] + new + text[pos + len(old):]


def run_mutant(tmp, idx, name, old, new, which):
    src = os.path.join(tmp, f"m{idx}.c")
    lib = os.path.join(tmp, f"libm{idx}.so")
    with open(SRC) as fh:
        text = fh.read()
    mutated = mutate(text, old, new, which)
    assert mutated != text
    with open(src, "w") as fh:
        fh.write(mutated)
    subprocess.run(["gcc"] + oracle.CFLAGS + ["-o", lib, src, "-lm"], check=True)
    env = dict(os.environ, OMP_NUM_THREADS="2")
    try:
        r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, lib, src], capture_output=True, text=True,
                           timeout=600, env=env)
    except subprocess.TimeoutExpired:
        return name, None, "timed out"
    return name, r.returncode, (r.stdout.strip() or r.stderr.strip()).splitlines()[-1:] or [""]


def test_every_mutant_fails_a_pin(tmp_path):
    with ThreadPoolExecutor(max_workers=4) as ex:
        res = list(ex.map(lambda a: run_mutant(str(tmp_path), *a),
                          [(i,) + m for i, m in enumerate(MUTANTS)]))
    survivors = [(name, out) for name, rc, out in res if rc == 0 or rc is None]
    assert not survivors, f"mutants no pin catches: {survivors}"


def test_unmutated_copy_passes_every_pin(tmp_path):
    # the runner itself: the oracle's own source, compiled the same way, survives
    src = os.path.join(str(tmp_path), "orig.c")
    lib = os.path.join(str(tmp_path), "liborig.so")
    with open(SRC) as fh, open(src, "w") as out:
        out.write(fh.read())
    subprocess.run(["gcc"] + oracle.CFLAGS + ["-o", lib, src, "-lm"], check=True)
    r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, lib, src], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "survived every pin" in r.stdout


# The oracle's Python wrapper (oracle/__init__.py), which marshals operands
# into the C code: the same check, with the wrapper's source mutated and the
# C library as built.  Occurrences of the repeated marshalling line follow
# the file: partials_I, emu_I, partials_F8, emu_F8, emu_II, dd_gemm.
WRAPPER_SRC = os.path.join(ROOT, "oracle", "__init__.py")
WRAPPER_MUTANTS = [
    ("emu_I takes B untransposed", "A, Bt = _f64(A), _f64(np.asarray(B).T)", "A, Bt = _f64(A), _f64(np.asarray(B))", 1),
    ("emu_II takes B untransposed", "A, Bt = _f64(A), _f64(np.asarray(B).T)", "A, Bt = _f64(A), _f64(np.asarray(B))", 4),
    ("dd_gemm takes B untransposed", "A, Bt = _f64(A), _f64(np.asarray(B).T)", "A, Bt = _f64(A), _f64(np.asarray(B))", 5),
    ("emu_Z3M conjugates B", "Bt = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).T)",
     "Bt = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).conj().T)", 0),
    ("dd_zgemm conjugates B", "Bt = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).T)",
     "Bt = np.ascontiguousarray(np.asarray(B, dtype=np.complex128).conj().T)", 2),
    ("emu_Z3M conjugates alpha", "alpha, beta = complex(alpha), complex(beta)",
     "alpha, beta = complex(alpha).conjugate(), complex(beta)", 0),
    ("emu_Z4M_I conjugates beta", "alpha, beta = complex(alpha), complex(beta)",
     "alpha, beta = complex(alpha), complex(beta).conjugate()", 1),
    ("column exponents of the rows of B", "return row_exponents(np.ascontiguousarray(np.asarray(B, dtype=np.float64).T))",
     "return row_exponents(np.ascontiguousarray(np.asarray(B, dtype=np.float64)))", None),
    ("complex residues with real-part exponents", "        E = row_exponents_z(X)\n", "        E = row_exponents(X.real)\n", None),
    ("error metric over |AB| instead of |A||B|", "den = np.abs(np.asarray(A)) @ np.abs(np.asarray(B))",
     "den = np.abs(np.asarray(A) @ np.asarray(B))", None),
]


def run_wrapper_mutant(tmp, idx, name, old, new, which):
    with open(WRAPPER_SRC) as fh:
        text = fh.read()
    wsrc = os.path.join(tmp, f"wrapper_m{idx}.py")
    with open(wsrc, "w") as fh:
        fh.write(mutate(text, old, new, which) if old is not None else text)
    lib = oracle.build()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    try:
        r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, lib, SRC, wsrc], capture_output=True, text=True,
                           timeout=600, env=env)
    except subprocess.TimeoutExpired:
        return name, None, "timed out"
    return name, r.returncode, (r.stdout.strip() or r.stderr.strip()).splitlines()[-1:] or [""]


def test_every_wrapper_mutant_fails_a_pin(tmp_path):
    with ThreadPoolExecutor(max_workers=4) as ex:
        res = list(ex.map(lambda a: run_wrapper_mutant(str(tmp_path), *a),
                          [(i,) + m for i, m in enumerate(WRAPPER_MUTANTS)]))
    survivors = [(name, out) for name, rc, out in res if rc == 0 or rc is None]
    assert not survivors, f"mutants no pin catches: {survivors}"
    name, rc, out = run_wrapper_mutant(str(tmp_path), "orig", "unmutated", None, None, None)
    assert rc == 0 and "survived" in out[0], out


# The selector oracle (oracle/selector.py, numpy): the same check against its
# pins in test_selector_oracle.py.  (Moving eps inside the square root of the
# Adam step is left out: it changes a step by about 5e-9 of itself.)
SELECTOR_SRC = os.path.join(ROOT, "oracle", "selector.py")
SELECTOR_MUTANTS = [
    ("cross-entropy gradient not averaged", "    dz3 /= b\n", "", None),
    ("softmax gradient sign", "dz3[np.arange(b), y] -= 1.0", "dz3[np.arange(b), y] += 1.0", None),
    ("W2 gradient transposed", 'g["W2"] = dz2.T @ h1', 'g["W2"] = (dz2.T @ h1).T', None),
    ("first ReLU not back-propagated", "dz1 = dh1 * (z1 > 0)", "dz1 = dh1", None),
    ("b1 gradient averaged", 'g["b1"] = dz1.sum(axis=0)', 'g["b1"] = dz1.mean(axis=0)', None),
    ("second layer without bias", 'z2 = h1 @ p["W2"].T + p["b2"]', 'z2 = h1 @ p["W2"].T', None),
    ("Adam second moment of |g|", "v = b2 * v + (1 - b2) * grad * grad", "v = b2 * v + (1 - b2) * np.abs(grad)", None),
    ("Adam without the second bias correction", "c2 = 1 - b2 ** step", "c2 = 1.0", None),
    ("feature bins of 4 exponents", "h[min(max(d, 0) // 3, 31)] += 1", "h[min(max(d, 0) // 4, 31)] += 1", None),
    ("zeros counted in bin 0", "h[31] += 1", "h[0] += 1", None),
    ("row exponent of the first element", "E = _frexp_exp(float(np.max(np.abs(row)))) if row.size else 0",
     "E = _frexp_exp(float(row[0])) if row.size else 0", None),
    ("features of the rows of B", "Bt = np.ascontiguousarray(np.asarray(B, dtype=np.float64).T)",
     "Bt = np.ascontiguousarray(np.asarray(B, dtype=np.float64))", None),
    ("K feature scale", "f[64] = np.float32(math.log2(k) / 16.0)", "f[64] = np.float32(math.log2(k) / 8.0)", None),
    ("tolerance feature sign", "f[65] = np.float32(-math.log10(tol) / 16.0)",
     "f[65] = np.float32(math.log10(tol) / 16.0)", None),
]

SELECTOR_RUNNER = r"""
import importlib.util, os, sys
root, src = sys.argv[1:3]
sys.path[:0] = [root, os.path.join(root, "tests")]
import oracle
spec = importlib.util.spec_from_file_location("oracle.selector", src)
mod = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mod)
sys.modules["oracle.selector"] = mod
oracle.selector = mod
import test_selector_oracle as T
for name in sorted(dir(T)):
    if name.startswith("test_"):
        try:
            getattr(T, name)()
        except Exception as e:
            print("caught by", name, type(e).__name__)
            sys.exit(1)
print("survived every pin")
sys.exit(0)
"""


def run_selector_mutant(tmp, idx, name, old, new, which):
    with open(SELECTOR_SRC) as fh:
        text = fh.read()
    src = os.path.join(tmp, f"selector_m{idx}.py")
    with open(src, "w") as fh:
        fh.write(mutate(text, old, new, which) if old is not None else text)
    r = subprocess.run([sys.executable, "-c", SELECTOR_RUNNER, ROOT, src], capture_output=True, text=True,
                       timeout=600)
    return name, r.returncode, (r.stdout.strip() or r.stderr.strip()).splitlines()[-1:] or [""]


def test_every_selector_mutant_fails_a_pin(tmp_path):
    with ThreadPoolExecutor(max_workers=4) as ex:
        res = list(ex.map(lambda a: run_selector_mutant(str(tmp_path), *a),
                          [(i,) + m for i, m in enumerate(SELECTOR_MUTANTS)]))
    survivors = [(name, out) for name, rc, out in res if rc == 0]
    assert not survivors, f"mutants no pin catches: {survivors}"
    # and the unmutated copy passes
    name, rc, out = run_selector_mutant(str(tmp_path), "orig", "unmutated", None, None, None)
    assert rc == 0 and "survived" in out[0], out


@pytest.mark.parametrize("i", range(len(MUTANTS)))
def test_mutation_site_is_unique_or_indexed(i):
    name, old, new, which = MUTANTS[i]
    with open(SRC) as fh:
        text = fh.read()
    if which is None:
        assert text.count(old) == 1, f"{name}: the site occurs {text.count(old)} times"
    else:
        assert text.count(old) > which, name
