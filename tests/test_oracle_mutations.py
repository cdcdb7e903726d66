"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source -- a wrong
bit in the Sobol recurrence, a transposed operand in the grid map, a missing
factor of the Jacobian, a dropped square in an integrand, a wrong neighbour
in the smoothing, a variance without its n-1, ... -- compiles it, runs the
pin tests against it, and requires at least one pin to fail.  (The copies
are test artefacts; the oracle itself is unchanged.)"""
import inspect

import pytest

import oracle as O

from . import test_oracle_genz as TG
from . import test_oracle_sobol as TS
from . import test_oracle_vegas as TV

MUTATIONS = [
    ("sobol recurrence shift", "mk ^= m[k - j] << j;", "mk ^= m[k - j] << (j + 1);"),
    ("gray code dropped", "uint64_t g = i ^ (i >> 1);", "uint64_t g = i;"),
    ("map operands transposed", "x[d] = fma(w, frac, e[k]);", "x[d] = fma(frac, w, e[k + 1]);"),
    ("jacobian without N", "J *= (double)nbins * w;", "J *= w;"),
    ("gaussian without square of a", "s += a[i] * a[i] * dx * dx;", "s += a[i] * dx * dx;"),
    ("c0 sign", "s += a[i] * fabs(x[i] - u[i]);", "s += a[i] * (x[i] - u[i]);"),
    ("corner peak exponent", "return pow(1.0 + s, -(double)(ndim + 1));", "return pow(1.0 + s, -(double)ndim);"),
    ("oscillatory phase", "return cos(2.0 * OR_PI * u[0] + s);", "return cos(OR_PI * u[0] + s);"),
    ("smoothing neighbour", "h[k] = (Hd[k - 1] + Hd[k] + Hd[k + 1]) / 3.0;", "h[k] = (Hd[k - 1] + Hd[k] + Hd[k]) / 3.0;"),
    ("compression exponent", "r[k] = q * sqrt(q); /* q^1.5 */", "r[k] = q * q;"),
    ("rebin interpolation", "e_new[m] = fma(e[k + 1] - e[k], (t - C[k]) / r[k], e[k]);",
     "e_new[m] = fma(e[k + 1] - e[k], (t - C[k]) / r[k], e[k + 1]);"),
    ("variance without n-1", "double var = (S2[c] / (double)nj - I * I) / (double)(nj - 1);",
     "double var = (S2[c] / (double)nj - I * I) / (double)nj;"),
    ("inverse-variance weights", "sum_add(&W, 1.0 / var[j]);", "sum_add(&W, 1.0 / sqrt(var[j]));"),
    ("chi2 odd dof", "Q = erfc(sqrt(z)) + exp(-z) * acc;", "Q = erfc(z) + exp(-z) * acc;"),
    ("histogram of component 1", "if (c == 0)\n                Jf0 = Jf;", "if (c == 1)\n                Jf0 = Jf;"),
    ("index 0 not skipped", "uint64_t next_index = 1;", "uint64_t next_index = 0;"),
]


def _pins():
    """Every pin test of the oracle with every parameter set."""
    import itertools
    out = []
    for mod in (TS, TV, TG):
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if not name.startswith("test_") or fn.__module__ != mod.__name__:
                continue
            if "tmp_path" in inspect.signature(fn).parameters:
                continue
            axes = []
            for m in getattr(fn, "pytestmark", []):
                if m.name == "parametrize":
                    names = [n.strip() for n in m.args[0].split(",")] if isinstance(m.args[0], str) else m.args[0]
                    axes.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in m.args[1]])
            for combo in itertools.product(*axes) if axes else [()]:
                kwargs = {}
                for part in combo:
                    kwargs.update(part)
                out.append((f"{mod.__name__}.{name}{kwargs}", fn, kwargs))
    return out


@pytest.mark.parametrize("label,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, label, old, new):
    src = O.source()
    assert src.count(old) == 1, f"mutation anchor not found: {label}"
    lib = O.compile_variant(src.replace(old, new), str(tmp_path / "libmut.so"))
    failed = []
    with O.use_library(lib):
        for name, fn, kwargs in _pins():
            try:
                fn(**kwargs)
            except Exception:
                failed.append(name)
                break
    assert failed, f"no pin caught: {label}"
