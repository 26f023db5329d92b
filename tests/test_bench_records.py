"""Host-side checks of what bench.py reports (no GPU).

The roofline's memory and issue views scale per-particle-step figures from a
committed ncu capture; bench.py uses them only while the advection kernel's
sources hash to the captured version.  These tests keep the committed capture
in step with the sources and check the figures it carries.
"""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_committed_capture_matches_the_kernel_sources():
    cap = bench.captured_traffic()
    assert cap is not None, (
        "profiles/advect_f32_3d_traffic.json was captured on other kernel sources "
        f"(hash now {bench.kernel_hash()}): take the capture again")


def test_capture_figures_are_consistent():
    d = json.load(open(os.path.join(ROOT, "profiles", "advect_f32_3d_traffic.json")))
    particle_steps = 2_000_000 * 48            # the captured case: 2M particles x 48 steps
    warp_steps = particle_steps / 32
    assert abs(d["dram_bytes_per_particle_step"]
               - (d["dram_bytes_read"] + d["dram_bytes_write"]) / particle_steps) < 1e-9
    assert abs(d["l2_bytes_per_particle_step"] - d["l2_bytes"] / particle_steps) < 1e-9
    assert abs(d["l1_bytes_per_particle_step"] - d["l1_bytes"] / particle_steps) < 1e-9
    assert 0 < d["warp_instructions_per_warp_step"] * warp_steps < 1e10
    # the register corner cache keeps DRAM far below the method's 810 B of gathers
    assert d["dram_bytes_per_particle_step"] < bench.ALGO_BYTES_PER_STEP / 10
