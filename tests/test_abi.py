"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU
and exports every entry point that include/itokmc.h declares; the binding's
struct layouts match the header's (compiled with gcc)."""
import ctypes
import os
import subprocess
import tempfile

import pytest

from paper_2307_01797_gb300 import build, itokmc


def test_library_exports_every_header_symbol():
    L = itokmc.lib()
    names = itokmc.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert b"sm_103a" in L.itokmc_version()


def test_config_defaults_without_gpu():
    c = itokmc.Config()
    assert itokmc.lib().itokmc_config_defaults(ctypes.byref(c)) == 0
    assert c.n_new == 64 and c.n_crit == 5 and c.n_ssa == 10 and c.frac_bits == 10
    assert c.mg_rtol == 1e-10 and c.eps == float("inf")


def test_init_rejects_bad_config_without_touching_the_gpu():
    c = itokmc.Config()
    itokmc.lib().itokmc_config_defaults(ctypes.byref(c))
    c.n[0] = c.n[1] = c.n[2] = 12          # not a power of two
    c.particle_capacity = 10
    h = ctypes.c_void_p()
    assert itokmc.lib().itokmc_init(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"power of two" in itokmc.lib().itokmc_last_error(None)


@pytest.mark.parametrize("prec,fprec", [(0, 2), (1, 7), (2, -1), (-1, 0)])
def test_init_rejects_unknown_precision_without_touching_the_gpu(prec, fprec):
    """Only ITOKMC_FP64 / ITOKMC_MIXED select a form (field_precision also -1:
    as precision); anything else is refused before any device work."""
    from paper_2307_01797_gb300 import synth
    c = itokmc.make_config(synth.physics_small(16), 1000)
    c.precision, c.field_precision = prec, fprec
    h = ctypes.c_void_p()
    assert itokmc.lib().itokmc_init(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"precision" in itokmc.lib().itokmc_last_error(None)


@pytest.mark.parametrize("prec,coupling", [(1, 1), (0, 2), (0, -1)])
def test_init_rejects_unsupported_coupling_without_touching_the_gpu(prec, coupling):
    """The semi-implicit step exists in the FP64 form; unknown couplings are refused."""
    from paper_2307_01797_gb300 import synth
    c = itokmc.make_config(synth.physics_small(16), 1000, precision=prec)
    c.coupling = coupling
    h = ctypes.c_void_p()
    assert itokmc.lib().itokmc_init(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"coupling" in itokmc.lib().itokmc_last_error(None)


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "itokmc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(itokmc_config), offsetof(itokmc_config, particle_capacity),
         offsetof(itokmc_config, alloc_ctx), offsetof(itokmc_config, field_precision),
         sizeof(itokmc_stats), offsetof(itokmc_stats, ms_field), offsetof(itokmc_config, blobs),
         offsetof(itokmc_config, ion_factor), sizeof(itokmc_seed_blob), offsetof(itokmc_seed_blob, realization),
         offsetof(itokmc_stats, dt_last), offsetof(itokmc_config, beta_np), offsetof(itokmc_stats, recombinations_np),
         offsetof(itokmc_config, D_ion), offsetof(itokmc_stats, outflow_ion_neg), offsetof(itokmc_config, graph_step),
         offsetof(itokmc_stats, graph_steps));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(build.ROOT, "include"), c, "-o", exe], check=True)
        got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    C, S = itokmc.Config, itokmc.Stats
    B = itokmc.SeedBlob
    assert got == [ctypes.sizeof(C), C.particle_capacity.offset, C.alloc_ctx.offset, C.field_precision.offset,
                   ctypes.sizeof(S), S.ms_field.offset, C.blobs.offset, C.ion_factor.offset, ctypes.sizeof(B),
                   B.realization.offset, S.dt_last.offset, C.beta_np.offset, S.recombinations_np.offset,
                   C.D_ion.offset, S.outflow_ion_neg.offset, C.graph_step.offset, S.graph_steps.offset]


def test_oracle_and_library_share_no_source():
    """The oracle and the CUDA path are independent: no include or import
    crosses between them."""
    csrc = os.path.join(build.HERE, "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    odir = os.path.join(build.ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith((".c", ".py")):
            txt = open(os.path.join(odir, f)).read()
            assert "csrc" not in txt and "itokmc.h" not in txt and "paper_2307_01797_gb300" not in txt, f
