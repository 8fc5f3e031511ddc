"""CPU checks of the C ABI library (no GPU calls): it builds, loads, exports
every symbol include/ptp.h declares, its struct layouts match the binding,
and the host-side validation of the set_* calls reports errors as codes."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ptp():
    from paper_2502_21013_gb300 import build
    build.build()
    from paper_2502_21013_gb300 import ptp as mod
    return mod


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "ptp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ptp_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(ptp):
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(ptp.lib, name), name
    assert set(names) == set(ptp.EXPORTED)


def test_abi_sizes_and_defaults(ptp):
    import ctypes
    so, ss = ctypes.c_size_t(), ctypes.c_size_t()
    ptp.lib.ptp_abi_sizes(ctypes.byref(so), ctypes.byref(ss))
    assert so.value == ctypes.sizeof(ptp.Opts) and ss.value == ctypes.sizeof(ptp.Stats)
    o = ptp.default_opts()
    assert o.tol == 1e-8 and o.precision == ptp.PTP_MIXED and o.spatial_prec == ptp.PTP_PREC_GMG
    assert b"sm_103a" in ptp.lib.ptp_version()


def test_host_side_validation_without_gpu(ptp):
    import workloads as W
    prob = W.unit_square_problem(9, 4)
    c = ptp.Context(0)
    with pytest.raises(ptp.PtpError) as e:
        c.set_materials(prob.sigma_e, prob.nonlinear_e, 1.0, 100.0, 1.0, 100.0)  # before the mesh
    assert e.value.code == ptp.PTP_EINVAL
    bad = prob.tri.copy()
    bad[0, 0] = prob.n_nodes
    with pytest.raises(ptp.PtpError):
        c.set_mesh(prob.xy, bad, prob.dirichlet)
    ptp.load_problem(c, prob)
    with pytest.raises(ptp.PtpError):
        c.set_materials(-prob.sigma_e - 1, prob.nonlinear_e, 1.0, 100.0, 1.0, 100.0)
    with pytest.raises(ptp.PtpError):
        c.set_materials(prob.sigma_e, prob.nonlinear_e, 1.0, 100.0, 0.0, 100.0)
    coil = prob.coil_of_elem.copy()
    coil[0] = 5
    with pytest.raises(ptp.PtpError):
        c.set_sources(coil, prob.amp, prob.phase)
    with pytest.raises(ptp.PtpError):
        c.set_time(1.0, 0)
    with pytest.raises(ptp.PtpError) as e:
        c.residual(np.zeros((49, 4)))
    assert e.value.code in (ptp.PTP_ESTATE, ptp.PTP_ECUDA)
    c.close()


def test_no_cpu_fallback_in_product_package():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2502_21013_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower() or f.endswith(".h"), f


def test_new_option_defaults(ptp):
    o = ptp.default_opts()
    assert o.coarse_solver == ptp.PTP_COARSE_VCYCLES and o.dft_max_it == 30
    assert o.init_static == 0 and o.init_tol == 0.0
    assert o.newton_eta == 1e-2 and o.krylov_dim == 20


def test_law_and_khat_validation_without_gpu(ptp):
    import workloads as W
    prob = W.paper_transformer_problem(11, 13, 4)
    c = ptp.Context(0)
    c.set_structured(*prob.grid)
    with pytest.raises(ptp.PtpError) as e:          # the law needs the materials first
        c.set_law_exp(prob.law_abcd)
    assert e.value.code == ptp.PTP_EINVAL
    c.set_materials(prob.sigma_e, prob.nonlinear_e, prob.nu_min, prob.nu_max, prob.s_sat, prob.nu_linear)
    c.set_law_exp(prob.law_abcd)
    bad = prob.law_abcd.copy()
    bad[np.flatnonzero(prob.nonlinear_e)[0], 2] = 0.5   # c < 1
    with pytest.raises(ptp.PtpError):
        c.set_law_exp(bad)
    c.set_law_exp(None)
    c.set_khat(prob.khat_e)
    k = prob.khat_e.copy()
    k[3] = -1.0
    with pytest.raises(ptp.PtpError):
        c.set_khat(k)
    c.set_khat(None)


def test_non_finite_inputs_and_array_lengths_are_rejected(ptp):
    import workloads as W
    prob = W.unit_square_problem(9, 4)
    c = ptp.Context(0)
    xy = prob.xy.copy()
    xy[3, 0] = np.nan
    with pytest.raises(ptp.PtpError):
        c.set_mesh(xy, prob.tri, prob.dirichlet)
    with pytest.raises(ptp.PtpError):
        c.set_structured(9, 9, 0.0, 0.0, np.inf, 1.0)
    with pytest.raises(ptp.PtpError):
        c.set_structured(1 << 15, 1 << 15, 0.0, 0.0, 1.0, 1.0)   # more than 2^28 nodes
    ptp.load_problem(c, prob)
    s = prob.sigma_e.copy()
    s[0] = np.inf
    with pytest.raises(ptp.PtpError):
        c.set_materials(s, prob.nonlinear_e, 1.0, 100.0, 1.0, 100.0)
    with pytest.raises(ptp.PtpError):
        c.set_materials(prob.sigma_e, prob.nonlinear_e, 1.0, np.inf, 1.0, 100.0)
    with pytest.raises(ptp.PtpError):
        c.set_time(np.inf, 4)
    amp = np.array(prob.amp, dtype=np.float64)
    amp[0] = np.nan
    with pytest.raises(ptp.PtpError):
        c.set_sources(prob.coil_of_elem, amp, prob.phase)
    # per-element arrays must match the mesh: the library reads n_tri entries
    with pytest.raises(ptp.PtpError) as e:
        c.set_materials(prob.sigma_e[:-1], prob.nonlinear_e[:-1], 1.0, 100.0, 1.0, 100.0)
    assert e.value.code == ptp.PTP_EINVAL
    with pytest.raises(ptp.PtpError):
        c.set_sources(prob.coil_of_elem[:-1], prob.amp, prob.phase)
    with pytest.raises(ptp.PtpError):
        c.set_sources(prob.coil_of_elem, prob.amp, np.zeros(len(prob.amp) + 1))
    with pytest.raises(ptp.PtpError):
        c.set_khat(np.ones(prob.n_tri + 1))
    with pytest.raises(ptp.PtpError):
        c.set_law_exp(np.ones((prob.n_tri, 3)))
    with pytest.raises(ptp.PtpError):
        c.set_mesh(prob.xy, prob.tri, prob.dirichlet[:-1])
    # the valid problem still loads after the rejected calls
    ptp.load_problem(c, prob)
    c.close()


def test_binding_checks_block_sizes_before_calling_the_library(ptp):
    """The library reads and writes n * (N >> level) values per block; the
    binding compares every array with that count first (sizes of a set-up
    context are faked here, since ptp_setup needs a GPU)."""
    torch = pytest.importorskip("torch")
    c = ptp.Context(0)
    c._sizes = (10, 8, 30, 3)          # n_free, N, n_tri, time levels
    assert [c._count(l) for l in range(4)] == [80, 40, 20, None]
    with pytest.raises(ptp.PtpError) as e:
        c.apply_shifted_dev(0, torch.zeros(10, 4), torch.zeros(10, 4))
    assert e.value.code == ptp.PTP_EINVAL and "80 elements" in str(e.value)
    with pytest.raises(TypeError):     # right size, but not a CUDA tensor
        c.apply_shifted_dev(1, torch.zeros(10, 4), torch.zeros(10, 4))
    for call in (lambda: c.solve_dev(torch.zeros(10, 7), ptp.default_opts()),
                 lambda: c.residual_dev(torch.zeros(10, 8), torch.zeros(81)),
                 lambda: c.spatial_solve_dev(2, torch.zeros(10, 4), torch.zeros(10, 4), 1e-6, 5),
                 lambda: c.periodic_solve_dev(torch.zeros(79), torch.zeros(80), 1),
                 lambda: c.jacobian_apply_dev(torch.zeros(8), torch.zeros(80), torch.zeros(80)),
                 lambda: c.loss_dev(torch.zeros(10, 9))):
        with pytest.raises(ptp.PtpError):
            call()
    with pytest.raises(ptp.PtpError) as e:
        c.residual(np.zeros((10, 7)))
    assert "expected 80 values" in str(e.value)
    with pytest.raises(ptp.PtpError) as e:
        c.solve(ptp.default_opts(), U_out=np.zeros((10, 8), dtype=np.float32))
    assert "float64" in str(e.value)
    c.set_time(1.0, 4)                 # any change of the problem forgets the sizes
    assert c._sizes is None and c._count() is None
    c.close()


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ptp.h"

int main(void) {
    ptp_opts o;
    size_t so = 0, ss = 0;
    ptp_ctx* ctx = NULL;
    ptp_default_opts(&o);
    ptp_abi_sizes(&so, &ss);
    if (so != sizeof(ptp_opts) || ss != sizeof(ptp_stats)) return 2;
    if (o.precision != PTP_MIXED || o.tol != 1e-8) return 3;
    if (ptp_create(&ctx, 0) != PTP_OK || ctx == NULL) return 4;
    if (ptp_set_time(ctx, -1.0, 4) != PTP_EINVAL) return 5;     /* host-side check, no GPU */
    if (strlen(ptp_last_error(ctx)) == 0) return 6;
    if (ptp_set_time(ctx, 0.02, 4) != PTP_OK) return 7;
    ptp_destroy(ctx);
    printf("%s\n", ptp_version());
    return 0;
}
"""


def test_header_is_c99_and_the_library_links_from_c(ptp):
    """include/ptp.h is plain C: a C99 program (-pedantic -Werror) compiles
    against it, links libptp and calls the host-only entry points."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    out = os.path.join(ROOT, "paper_2502_21013_gb300", "_build", "c_abi_check")
    os.makedirs(out, exist_ok=True)
    src, exe = os.path.join(out, "main.c"), os.path.join(out, "main")
    with open(src, "w") as fh:
        fh.write(C_PROGRAM)
    libdir = os.path.dirname(ptp.LIB_PATH)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), src, "-o", exe,
                        "-L", libdir, "-lptp", "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert "sm_103a" in r.stdout
