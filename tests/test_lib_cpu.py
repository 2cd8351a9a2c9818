"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point declared in include/pod.h, validates parameters and
computes the POD basis on the host (compared with the oracle's own basis)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2212_14446_gb300 import build as b
    b.build()
    import paper_2212_14446_gb300 as p
    p.lib()
    return p


def header_symbols():
    with open(os.path.join(ROOT, "include", "pod.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(pod_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(pkg):
    syms = header_symbols()
    assert "pod_create" in syms and "pod_energy_forces" in syms and "pod_fit" in syms
    L = pkg.lib()
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(pkg.EXPORTS) == syms


def test_binding_constants_match_header(pkg):
    """Every #define POD_* integer of include/pod.h has the same value in the binding."""
    with open(os.path.join(ROOT, "include", "pod.h")) as f:
        text = f.read()
    defs = re.findall(r"^#define (POD_\w+) \(?(-?\d+)\)?", text, re.M)
    assert len(defs) >= 20
    for name, val in defs:
        assert hasattr(pkg, name), name
        assert getattr(pkg, name) == int(val), name


def test_workspace_limit_option(pkg):
    """POD_OPT_WORKSPACE_LIMIT_MB takes a cap >= 0 (0: none); a negative one is refused."""
    pod = pkg.POD(synth.params_small())
    pod.set_workspace_limit_mb(16)
    pod.set_workspace_limit_mb(0)
    with pytest.raises(pkg.PodError) as ei:
        pod.set_workspace_limit_mb(-1)
    assert ei.value.code == pkg.POD_EINVAL


def test_library_links_no_oracle(pkg):
    # the product library must not contain or reference any oracle symbol
    with open(pkg.LIB_PATH, "rb") as f:
        blob = f.read()
    assert b"orc_" not in blob


def test_param_validation(pkg):
    good = synth.params_full()
    bad_cases = [dict(r_in=5.0, r_cut=1.0), dict(beta=[0.0]), dict(P3=7), dict(K2=40), dict(alpha=[1.0] * 9),
                 dict(K2=0, K3=0, K4=0), dict(K2=20, K3=1, K4=1)]
    for kw in bad_cases:
        p = synth.PODParams(**{**good.__dict__, **kw})
        with pytest.raises(pkg.PodError) as ei:
            pkg.POD(p)
        assert ei.value.code == pkg.POD_EINVAL


def test_selftest_wait_validates_arguments(pkg):
    # refused before any CUDA call, so this runs without a GPU
    for limit in (-1, 10**10 + 1):
        with pytest.raises(pkg.PodError) as ei:
            pkg.pod_selftest_wait(limit)
        assert ei.value.code == pkg.POD_EINVAL


def test_sizes_match_oracle(pkg):
    for p in (synth.params_small(), synth.params_full(),
              synth.PODParams(K2=2, K3=1, K4=1, P3=2, P4=1), synth.PODParams(K2=5, K3=3, K4=3, P3=2, P4=2)):
        pod = pkg.POD(p)
        o = oracle.Oracle(p)
        assert (pod.M, pod.Ns, pod.K) == (o.M, o.Ns, o.K)


@pytest.mark.parametrize("which", ["small", "full"])
def test_basis_matches_oracle(pkg, which):
    """The library's POD (one-sided Jacobi on the snapshot matrix) and the
    oracle's (cyclic Jacobi on the Gram matrix) are different algorithms for the
    same eigenvectors; they agree to eigenvector perturbation accuracy,
    eps * lambda_1 / gap ~ 1e-12 relative here."""
    p = synth.params_small() if which == "small" else synth.params_full()
    pod = pkg.POD(p)
    o = oracle.Oracle(p)
    K = o.K
    lam = o.eig
    gaps = np.array([min(lam[k - 1] - lam[k] if k else np.inf, lam[k] - lam[k + 1]) for k in range(K)])
    bound = 1e3 * np.finfo(float).eps * lam[0] / gaps  # per-mode relative bound with a safety factor
    err = np.max(np.abs(pod.Q - o.Q), axis=0) / np.max(np.abs(o.Q), axis=0)
    assert np.all(err <= np.maximum(bound, 1e-13)), (err, bound)
    assert np.allclose(pod.eig[:K], lam[:K], rtol=1e-9)


def test_user_Q_override(pkg):
    p = synth.params_full()
    o = oracle.Oracle(p)
    Q = o.Q * 1.0
    pod = pkg.POD(p, Q=Q)
    assert np.array_equal(pod.Q, Q)


def test_model_file_round_trip(pkg, tmp_path):
    """pod_save / pod_load: parameters, Q and c come back bit for bit; a file
    without coefficients loads with none; no temporary file is left behind."""
    p = synth.params_full()
    pod = pkg.POD(p, precision="mixed")
    c = synth.coefficients(pod.M, 141)
    path = tmp_path / "ta.pod"
    pod.save(str(path), c)
    assert sorted(x.name for x in tmp_path.iterdir()) == ["ta.pod"]
    pod2, c2 = pkg.POD.load(str(path), "mixed")
    assert (pod2.M, pod2.Ns, pod2.K) == (pod.M, pod.Ns, pod.K)
    assert np.array_equal(pod2.Q, pod.Q) and np.array_equal(c2, c)
    pod.save(str(path))  # overwrite, no coefficients
    pod3, c3 = pkg.POD.load(str(path), "fp64")
    assert c3 is None and np.array_equal(pod3.Q, pod.Q)
    small = pkg.POD(synth.params_small())
    small.save(str(tmp_path / "small.pod"), synth.coefficients(small.M, 142))
    pod4, c4 = pkg.POD.load(str(tmp_path / "small.pod"))
    assert pod4.M == small.M and np.array_equal(c4, synth.coefficients(small.M, 142))


def test_model_file_errors(pkg, tmp_path):
    with pytest.raises(pkg.PodError) as ei:
        pkg.POD.load(str(tmp_path / "missing.pod"))
    assert ei.value.code == pkg.POD_EIO
    bad = tmp_path / "bad.pod"
    bad.write_text("fastpod-model 1\nr_in 1\nr_cut oops\n")
    with pytest.raises(pkg.PodError) as ei:
        pkg.POD.load(str(bad))
    assert ei.value.code == pkg.POD_EINVAL
    pod = pkg.POD(synth.params_full())
    good = tmp_path / "good.pod"
    pod.save(str(good), synth.coefficients(pod.M, 143))
    text = good.read_text().replace("c 103", "c 102", 1)  # coefficient count off by one
    bad.write_text(text)
    with pytest.raises(pkg.PodError) as ei:
        pkg.POD.load(str(bad))
    assert ei.value.code == pkg.POD_EINVAL
    with pytest.raises(pkg.PodError) as ei:
        pod.save(str(tmp_path / "nan.pod"), np.full(pod.M, np.nan))
    assert ei.value.code == pkg.POD_EINVAL
    with pytest.raises(pkg.PodError) as ei:
        pod.save(str(tmp_path / "no_such_dir" / "x.pod"))
    assert ei.value.code == pkg.POD_EIO
