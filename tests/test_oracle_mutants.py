"""Planted mistakes in the oracle are caught by its pins (CPU only).

Each mutant is ``oracle/ebe_oracle.c`` with one plausible mistake -- a dropped
term or factor, a wrong sign, a wrong index, a wrong constant, a step left
out -- compiled into a library of its own.  The pin tests
(``tests/test_oracle_pins.py``) then run against it in a subprocess and must
fail; the unmodified source, compiled the same way, must pass them.  The
learned-preconditioner oracle ``oracle/mpnn.py`` is treated the same way: a
mutated copy is imported in place of the module before its pins
(``tests/test_mpnn_oracle.py``) run; so is the Python layer of the oracle
(``oracle/__init__.py``: wrappers, Dirichlet lift, Chebyshev roots), as a
mutated copy of the whole package placed first on the import path.  The mistakes are planted in copies
under pytest's temporary directory; the oracle itself is never changed.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ebe_oracle.c")
MPNN_SRC = os.path.join(ROOT, "oracle", "mpnn.py")

# (name, exact text in ebe_oracle.c, replacement); each text occurs once.
MUTANTS = [
    # element matrices, Eq. matrices_K_M
    ("K_e without the element measure", "Ke[i + nb * j] = vol * s;", "Ke[i + nb * j] = s;"),
    ("K_e with a wrong gradient index", "s += g[i * dim + d] * g[j * dim + d];", "s += g[i * dim + d] * g[i * dim + d];"),
    ("M_e with a wrong quadrature weight", "Me[i + nb * j] = vol / nq * m;", "Me[i + nb * j] = vol / (nq + 1) * m;"),
    ("M_e by the vertex rule (lumped)", "qp[q][i] = (i == q) ? 0.0 : 0.5;", "qp[q][i] = (i == q) ? 1.0 : 0.0;"),
    ("M_e with a wrong 3D quadrature point",
     "double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;",
     "double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(3.0)) / 20.0;"),
    ("Gauss-Jordan elimination with a wrong sign", "for (int c = 0; c < 2 * nb; ++c) V[k][c] -= fac * V[col][c];",
     "for (int c = 0; c < 2 * nb; ++c) V[k][c] += fac * V[col][c];"),
    ("tetrahedron volume without 1/3!", "double fact = (dim == 2) ? 2.0 : 6.0;", "double fact = (dim == 2) ? 2.0 : 2.0;"),
    ("gradients read from the wrong half of inv(V)", "grad[i * dim + d] = V[1 + d][nb + i];",
     "grad[i * dim + d] = V[1 + d][i];"),
    # local systems, Sec. 2
    ("A_e = K_e - nu M_e", "Ae[t] = Ke[t] + nu * Me[t];", "Ae[t] = Ke[t] - nu * Me[t];"),
    ("b_e with a wrong node index", "s += Me[i + nb * j] * f_nodal[elems[e * nb + j]];",
     "s += Me[i + nb * j] * f_nodal[elems[e * nb + i]];"),
    # Algorithm 1
    ("local residual with a wrong sign", "re[i] = (be ? be[e * nb + i] : 0.0) - s;", "re[i] = (be ? be[e * nb + i] : 0.0) + s;"),
    ("local product with a wrong index", "for (int j = 0; j < nb; ++j) s += Ae[i + nb * j] * xe[j];\n            re[i]",
     "for (int j = 0; j < nb; ++j) s += Ae[i + nb * j] * xe[i];\n            re[i]"),
    ("assembly overwrites instead of adding", "for (int i = 0; i < nb; ++i) r[idx[i]] += re[i];",
     "for (int i = 0; i < nb; ++i) r[idx[i]] = re[i];"),
    ("residual without r(nd) = 0", "    zero_rows(r, nd, n_d);\n}", "}"),
    ("operator with a wrong sign", "            y[idx[i]] += s;", "            y[idx[i]] -= s;"),
    ("operator without the Dirichlet mask", "    zero_rows(y, nd, n_d);\n}", "}"),
    ("load assembly overwrites", "for (int i = 0; i < nb; ++i) b[elems[e * nb + i]] += be[e * nb + i];",
     "for (int i = 0; i < nb; ++i) b[elems[e * nb + i]] = be[e * nb + i];"),
    ("Jacobi diagonal takes the first column", "d[elems[e * nb + i]] += A[(int64_t)nb * nb * e + i + nb * i];",
     "d[elems[e * nb + i]] += A[(int64_t)nb * nb * e + i];"),
    ("dense assembly onto the diagonal", "dense[(int64_t)idx[i] * n_n + idx[j]] += Ae[i + nb * j];",
     "dense[(int64_t)idx[i] * n_n + idx[i]] += Ae[i + nb * j];"),
    # Jacobi-PCG
    ("PCG beta inverted", "double beta = rho_new / rho;", "double beta = rho / rho_new;"),
    ("PCG residual update with a wrong sign", "x[i] += alpha * p[i]; r[i] -= alpha * q[i];",
     "x[i] += alpha * p[i]; r[i] += alpha * q[i];"),
    ("PCG without the Jacobi preconditioner in the loop",
     "for (int64_t i = 0; i < n_n; ++i) z[i] = dinv[i] * r[i];\n        double rho_new",
     "for (int64_t i = 0; i < n_n; ++i) z[i] = r[i];\n        double rho_new"),
    ("PCG step length halved", "double alpha = rho / pq;", "double alpha = 0.5 * rho / pq;"),
    ("PCG direction without the previous direction", "p[i] = z[i] + beta * p[i];", "p[i] = z[i];"),
    ("relative residual measured on x0", "double num = sqrt(dot(n_n, r, r));", "double num = den;"),
    # stationary iterations
    ("Richardson step with a wrong sign", "for (int64_t i = 0; i < n_n; ++i) x[i] += omega * r[i];",
     "for (int64_t i = 0; i < n_n; ++i) x[i] -= omega * r[i];"),
    ("two-level Chebyshev multiplies by the root", "for (int64_t i = 0; i < n_n; ++i) x[i] += r[i] / a;",
     "for (int64_t i = 0; i < n_n; ++i) x[i] += r[i] * a;"),
    ("two-level Chebyshev always takes the first root", "double a = alphas[k % N];", "double a = alphas[0];"),
    ("three-level first step as printed, 2/(l2-l1)", "x[i] += 2.0 / (l1 + l2) * r[i];", "x[i] += 2.0 / (l2 - l1) * r[i];"),
    ("recurrence of Eq. recrCk with a wrong sign", "double ratio_next = 2.0 * s - rho;", "double ratio_next = 2.0 * s + rho;"),
    ("three-level residual factor 2 instead of 4",
     "x[i] = xk + c_km1_over_c_kp1 * (xk - xprev[i]) + 4.0 / (l2 - l1) * c_k_over_c_kp1 * r[i];",
     "x[i] = xk + c_km1_over_c_kp1 * (xk - xprev[i]) + 2.0 / (l2 - l1) * c_k_over_c_kp1 * r[i];"),
    ("three-level ratio not advanced", "rho = c_k_over_c_kp1;", "rho = rho;"),
    ("C_1 inverted", "double rho = 1.0 / s;", "double rho = s;"),
    # discrete L2 error
    ("mass norm with a wrong index", "s += err[idx[i]] * Me[i + nb * j] * err[idx[j]];",
     "s += err[idx[i]] * Me[i + nb * j] * err[idx[i]];"),
    ("mass norm squared", "return sqrt(s);\n}", "return s;\n}"),
]


def _env(**extra):
    """The subprocesses' environment: the repository on the import path and one
    BLAS thread each (several pin runs go at once)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", **extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    return env


def _compile(src_text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", c, "-o", so, "-lm"], check=True)
    return so


def _run_pins(lib):
    env = _env(EBE_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                           "-p", "no:cacheprovider", "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=600)


def _source():
    with open(SRC) as f:
        return f.read()


def test_unmodified_copy_passes_the_pins(tmp_path):
    res = _run_pins(_compile(_source(), str(tmp_path), "control"))
    assert res.returncode == 0, res.stdout[-2000:]


def _run_c_mutant(d, old, new):
    return _run_pins(_compile(_source().replace(old, new), d, "mutant"))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(mutant_runs, name, old, new):
    assert _source().count(old) == 1, name
    res = mutant_runs[("c", name)]
    assert res.returncode == 1, (name, res.stdout[-2000:])   # 1: some pin failed (not a crash or a usage error)


# (name, exact text in mpnn.py, replacement); each text occurs once.
MPNN_MUTANTS = [
    ("graph keeps self loops", "keep = a != b", "keep = a == a"),
    ("neighbour sum instead of mean", "return sums / deg[:, None]", "return sums"),
    ("transposed mean without 1/deg", "np.add.at(out, idx, g[rows] / deg[rows, None])", "np.add.at(out, idx, g[rows])"),
    ("message with a wrong sign", "a = _mean_nbr(graph, h) - h", "a = _mean_nbr(graph, h) + h"),
    ("layer without the skip connection", "h = rd(h + np.maximum(v, 0.0))", "h = rd(np.maximum(v, 0.0))"),
    ("output without the Jacobi term", "z = np.where(free, zj + sz * o, 0.0)", "z = np.where(free, sz * o, 0.0)"),
    ("output scaled by rms(r)", "z = np.where(free, zj + sz * o, 0.0)", "z = np.where(free, zj + s * o, 0.0)"),
    ("second feature scaled by rms(r)", "x = np.stack([r / s, zj / sz], 1)", "x = np.stack([r / s, zj / s], 1)"),
    ("Dirichlet rows not zeroed", "z = np.where(free, zj + sz * o, 0.0)", "z = zj + sz * o"),
    ("backward ignores the relu gate", "gv = gh * (cache[\"vs\"][l] > 0.0)", "gv = gh"),
    ("backward drops the -h of the message", "gh = gh + gu[:, :H] - ga + _mean_nbr_T(graph, ga)",
     "gh = gh + gu[:, :H] + _mean_nbr_T(graph, ga)"),
    ("backward drops the skip connection", "gh = gh + gu[:, :H] - ga + _mean_nbr_T(graph, ga)",
     "gh = gu[:, :H] - ga + _mean_nbr_T(graph, ga)"),
    ("backward uses the transposed input weights", "g[\"W_in\"] = gh.T @ cache[\"x\"]",
     "g[\"W_in\"] = (cache[\"x\"].T @ gh).T[:, ::-1]"),
    ("loss gradient without the factor 2", "return float(w @ Aw) / eAe, -2.0 * Aw / eAe",
     "return float(w @ Aw) / eAe, -1.0 * Aw / eAe"),
    ("BF16 rounds half up", "bias = 0x7FFF + ((bits >> 16) & 1)", "bias = 0x8000"),
    ("BF16 truncates", "out = ((bits + bias) & 0xFFFF0000).astype(np.uint32)", "out = (bits & 0xFFFF0000).astype(np.uint32)"),
    ("FCG direction with a wrong sign", "p = z - (z @ q) / (p @ q) * p", "p = z + (z @ q) / (p @ q) * p"),
    ("FCG step from p.p", "al = (p @ r) / (p @ q)", "al = (p @ p) / (p @ q)"),
]

_MPNN_DRIVER = (
    "import importlib.util, sys\n"
    "spec = importlib.util.spec_from_file_location('oracle.mpnn', sys.argv[1])\n"
    "mod = importlib.util.module_from_spec(spec)\n"
    "sys.modules['oracle.mpnn'] = mod\n"
    "spec.loader.exec_module(mod)\n"
    "import oracle\n"
    "oracle.mpnn = mod\n"
    "import pytest\n"
    "sys.exit(pytest.main([sys.argv[2], '-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu']))\n"
)


def _run_mpnn_pins(path):
    env = _env()
    return subprocess.run([sys.executable, "-c", _MPNN_DRIVER, path, os.path.join(ROOT, "tests", "test_mpnn_oracle.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def _mpnn_source():
    with open(MPNN_SRC) as f:
        return f.read()


def test_unmodified_mpnn_copy_passes_the_pins(tmp_path):
    path = os.path.join(str(tmp_path), "mpnn_copy.py")
    with open(path, "w") as f:
        f.write(_mpnn_source())
    res = _run_mpnn_pins(path)
    assert res.returncode == 0, res.stdout[-2000:]


def _run_mpnn_mutant(d, old, new):
    path = os.path.join(d, "mpnn_mutant.py")
    with open(path, "w") as f:
        f.write(_mpnn_source().replace(old, new))
    return _run_mpnn_pins(path)


@pytest.mark.parametrize("name,old,new", MPNN_MUTANTS, ids=[m[0] for m in MPNN_MUTANTS])
def test_planted_mpnn_mistake_is_caught(mutant_runs, name, old, new):
    assert _mpnn_source().count(old) == 1, name
    res = mutant_runs[("mpnn", name)]
    assert res.returncode == 1, (name, res.stdout[-2000:])


# (name, exact text in oracle/__init__.py, replacement); each text occurs once.
PKG_MUTANTS = [
    ("Dirichlet values not carried by the iterate", "x[self.nd] = self.g", "x[self.nd] = 0.0"),
    ("default x0 of the relative residual without g", "x0 = self.with_dirichlet(np.zeros(self.n_n))",
     "x0 = np.zeros(self.n_n)"),
    ("PCG ignores the given x0", "x = self.with_dirichlet(np.zeros(self.n_n) if x0 is None else x0)",
     "x = self.with_dirichlet(np.zeros(self.n_n))"),
    ("PCG status codes swapped", '{0: "converged", 1: "maxit", 2: "breakdown"}', '{0: "maxit", 1: "converged", 2: "breakdown"}'),
    ("PCG info fields swapped", '"iterations": int(info[0]), "rel_residual": float(info[1]),',
     '"iterations": int(info[1]), "rel_residual": float(info[0]),'),
    ("dense K and M swapped", 'src = {"A": self._Ab, "K": self._Kb, "M": self._Mb}[which]',
     'src = {"A": self._Ab, "K": self._Mb, "M": self._Kb}[which]'),
    ("nu ignored", 'self.nu = float(prob["nu"])', "self.nu = 1.0"),
    ("Chebyshev roots: centre and half-width swapped", "d, c = 0.5 * (lam1 + lam2), 0.5 * (lam2 - lam1)",
     "d, c = 0.5 * (lam2 - lam1), 0.5 * (lam1 + lam2)"),
    ("Chebyshev roots at the wrong angles", "math.cos(math.pi * (k + 0.5) / N)", "math.cos(math.pi * (k + 1.0) / N)"),
]


def _copy_package(dst_root, text):
    import shutil
    pkg = os.path.join(dst_root, "oracle")
    os.makedirs(pkg)
    for name in ("ebe_oracle.c", "mpnn.py"):
        shutil.copy(os.path.join(ROOT, "oracle", name), os.path.join(pkg, name))
    with open(os.path.join(pkg, "__init__.py"), "w") as f:
        f.write(text)


def _run_pins_with_package(dst_root):
    env = _env()
    env.pop("EBE_ORACLE_LIB", None)
    env["PYTHONPATH"] = dst_root + os.pathsep + env["PYTHONPATH"]
    # run from the copy's directory: `python -c` puts the working directory
    # first on the import path; exit code 3 if the copy was not the one imported
    code = ("import sys, oracle, pytest\n"
            "if not oracle.__file__.startswith(sys.argv[1]): sys.exit(3)\n"
            "sys.exit(pytest.main([sys.argv[2], '-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu']))\n")
    return subprocess.run([sys.executable, "-c", code, dst_root, os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          cwd=dst_root, env=env, capture_output=True, text=True, timeout=600)


def _package_source():
    with open(os.path.join(ROOT, "oracle", "__init__.py")) as f:
        return f.read()


def test_unmodified_package_copy_passes_the_pins(tmp_path):
    _copy_package(str(tmp_path), _package_source())
    res = _run_pins_with_package(str(tmp_path))
    assert res.returncode == 0, res.stdout[-2000:] + res.stderr[-2000:]


def _run_pkg_mutant(d, old, new):
    _copy_package(d, _package_source().replace(old, new))
    return _run_pins_with_package(d)


@pytest.mark.parametrize("name,old,new", PKG_MUTANTS, ids=[m[0] for m in PKG_MUTANTS])
def test_planted_package_mistake_is_caught(mutant_runs, name, old, new):
    assert _package_source().count(old) == 1, name
    res = mutant_runs[("pkg", name)]
    assert res.returncode == 1, (name, res.stdout[-2000:], res.stderr[-2000:])


@pytest.fixture(scope="module")
def mutant_runs(tmp_path_factory):
    """Every mutant's pin run, each in its own directory and process, several
    at a time on a thread pool; keyed by (kind, name)."""
    jobs = ([("c", m, _run_c_mutant) for m in MUTANTS] + [("mpnn", m, _run_mpnn_mutant) for m in MPNN_MUTANTS]
            + [("pkg", m, _run_pkg_mutant) for m in PKG_MUTANTS])
    assert len({(kind, m[0]) for kind, m, _ in jobs}) == len(jobs), "mutant names must be unique"
    dirs = [str(tmp_path_factory.mktemp("mutant")) for _ in jobs]
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = {(kind, m[0]): ex.submit(fn, d, m[1], m[2]) for (kind, m, fn), d in zip(jobs, dirs)}
        return {key: f.result() for key, f in futs.items()}
