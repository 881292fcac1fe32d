"""Host-only: every workload program specialises and compiles for sm_103a (no device needed)."""
import pytest

import paper_2512_12615_gb300 as gx
from tests.asmtext import assemble
from workloads import programs as P


def _check(prog, specs, cs, det=True):
    rc, log = gx.jit_check(prog, specs, cs, deterministic=det)
    if rc == gx.E_NODEV:
        pytest.skip("no runtime compiler on this host")
    assert rc == 0, log


@pytest.mark.parametrize("build", [P.counting, P.page_heat, P.latency])
def test_workload_programs_compile(build):
    _check(*build())


@pytest.mark.parametrize("p", [0, 21, 63])
def test_batch_programs_compile(p):
    _check(*P.batch_programs()[p])


def test_rejected_program_is_not_compiled():
    rc, log = gx.jit_check(assemble(["ldx8 r0 r10 -8", "exit"]).prog(), [], 16)
    assert rc == gx.E_VERIFY and "uninitialised stack" in log
