"""The C-ABI library builds, loads and exports what include/neat.h declares.

CPU only: these tests make no CUDA call that needs a device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2404_01817_gb300 import build
    return build.build()


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^NEAT_API[^(]*?\b(neat_\w+)\s*\(", text, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = set(declared_symbols())
    for required in ("neat_transform", "neat_forward", "neat_transformed_bytes", "neat_forward_steps",
                     "neat_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib_path):
    from paper_2404_01817_gb300 import neat
    d = neat.dims(27, 8, 50, 200)
    stride = neat.neat_record_stride(d)
    assert stride % 128 == 0 and stride >= 32 + 16 * 50 + 8 * 200
    assert neat.neat_transformed_bytes(10000, d) == 10000 * stride
    assert neat.neat_record_stride(neat.dims(0, 1, 1025, 4)) == 0          # too many nodes
    assert neat.neat_record_stride(neat.dims(3, 0, 10, 4)) == 0            # no outputs
    assert neat.neat_record_stride(neat.dims(8, 4, 10, 4)) == 0            # I + O > Nmax
    assert neat.neat_record_stride(neat.dims(1, 1, 4, 8193)) == 0          # too many conns
    for B in (1, 2, 4, 17, 64, 256):
        for N in (10, 50, 100, 256, 300, 511, 1024):
            L = neat.neat_default_launch(1000, neat.dims(4, 2, N, 4 * N), B)
            assert L.group >= L.tile and L.group * L.groups_per_block <= 1024
            assert L.group & (L.group - 1) == 0 and L.tile & (L.tile - 1) == 0     # the kernels index by shifts


def test_argument_errors_do_not_touch_the_device(lib_path):
    from paper_2404_01817_gb300 import neat
    lib = neat._lib
    d = neat.dims(3, 1, 10, 20)
    assert lib.neat_transform(None, None, 4, d, None, 0, None, None) == neat.NEAT_EINVAL
    assert "null" in neat.last_error()
    assert lib.neat_transform(None, None, 4, neat.dims(3, 1, 2000, 20), None, 0, None, None) == neat.NEAT_EINVAL
    assert lib.neat_transform(16, 16, 4, d, 16, 10, None, None) == neat.NEAT_ENOMEM
    bad = neat.Launch(3, 1, 1, 0)
    assert lib.neat_forward_ex(16, 1, d, 16, 1, 16, ctypes.byref(bad), None) == neat.NEAT_EINVAL
    assert lib.neat_transform(None, None, 0, d, None, 0, None, None) == neat.NEAT_OK   # empty population


def test_argument_errors_of_the_other_entry_points(lib_path):
    """Sizes and argument checks of the recurrent, distance, evolve and
    substrate entry points, all answered on the host."""
    from paper_2404_01817_gb300 import neat
    lib = neat._lib
    d = neat.dims(27, 8, 50, 200)
    # sizes
    assert neat.neat_gene_stride(d) % 128 == 0
    assert neat.neat_gene_stride(d) >= 16 + 4 * 50 + 16 * 50 + 16 * 200
    assert neat.neat_gene_stride(neat.dims(0, 1, 1025, 4)) == 0
    assert neat.neat_mutation_sizes(d) == (16 + 6 * 50 + 2 * 200, 4 + 2 * 50 + 200)
    # empty work is a no-op, bad sizes and null pointers are NEAT_EINVAL
    assert lib.neat_transform_recurrent(None, None, 0, d, None, 0, None, None) == neat.NEAT_OK
    assert lib.neat_transform_recurrent(None, None, 4, d, None, 0, None, None) == neat.NEAT_EINVAL
    assert lib.neat_forward_recurrent(16, 1, d, 16, 1, -1, 16, None) == neat.NEAT_EINVAL
    assert lib.neat_distance_prepare(None, None, 0, d, None, 0, None, None) == neat.NEAT_OK
    assert lib.neat_distance_prepare(None, None, 3, d, None, 0, None, None) == neat.NEAT_EINVAL
    assert lib.neat_distance(16, 4, 16, 0, d, ctypes.c_float(1.0), ctypes.c_float(0.5), 16, 0, None) == neat.NEAT_OK
    assert lib.neat_distance(16, 4, 16, 5, d, ctypes.c_float(1.0), ctypes.c_float(0.5), 16, 4, None) \
        == neat.NEAT_EINVAL                                                   # ld_out < pop_b
    assert lib.neat_distance(16, 4, 24, 5, d, ctypes.c_float(1.0), ctypes.c_float(0.5), 16, 5, None) \
        == neat.NEAT_EINVAL                                                   # misaligned records
    assert lib.neat_speciate(16, 4, 8, 4, ctypes.c_float(3.0), 16, None) == neat.NEAT_EINVAL   # ld < n_reps
    assert lib.neat_speciate(None, 0, 8, 8, ctypes.c_float(3.0), None, None) == neat.NEAT_OK
    m = neat.mutation(node_add=0.2)
    assert lib.neat_mutate(None, None, 0, d, ctypes.byref(m), None, None, None, None) == neat.NEAT_OK
    assert lib.neat_mutate(16, 16, 2, d, ctypes.byref(m), None, 16, 16, None) == neat.NEAT_EINVAL
    m.n_activation_options = 9
    assert lib.neat_mutate(16, 16, 2, d, ctypes.byref(m), 16, 16, 16, None) == neat.NEAT_EINVAL
    assert lib.neat_crossover(16, 16, 4, d, 16, 0, 16, 16, 16, None) == neat.NEAT_OK
    assert lib.neat_crossover(16, 24, 4, d, 16, 2, 16, 16, 16, None) == neat.NEAT_EINVAL   # misaligned conns
    assert lib.neat_fill_words(1, 2, None, 0, None) == neat.NEAT_OK
    assert lib.neat_fill_words(1, 2, None, 8, None) == neat.NEAT_EINVAL
    assert lib.neat_substrate_forward(16, 4, neat.Substrate(1, 3), 16, 1, 1, 1, 16, None) == neat.NEAT_EINVAL
    assert lib.neat_substrate_forward(16, 4, neat.Substrate(16, 3), 16, 1, 9, 1, 16, None) == neat.NEAT_EINVAL
    assert lib.neat_substrate_forward(None, 0, neat.Substrate(16, 3), None, 1, 1, 1, None, None) == neat.NEAT_OK


def test_lane_program_sizes_and_argument_errors(lib_path):
    """Lane programs: buffer sizes and the argument checks of
    neat_lanes_pack / neat_forward_lanes, all answered on the host."""
    from paper_2404_01817_gb300 import neat
    lib = neat._lib
    d = neat.dims(27, 8, 50, 200)
    n = neat.neat_lanes_bytes(10000, d)
    assert n > 0 and n % 128 == 0
    assert neat.neat_lanes_bytes(10016, d) > n                     # one more warp of 16 genomes
    assert neat.neat_lanes_bytes(0, d) > 0                         # the header
    assert neat.neat_lanes_bytes(-1, d) == 0
    assert neat.neat_lanes_bytes(10, neat.dims(8, 4, 129, 200)) == 0    # more than 128 nodes
    assert neat.neat_lanes_bytes(10, neat.dims(8, 4, 128, 2000)) == 0   # a record above 12 KB
    assert neat.neat_lanes_bytes(10, neat.dims(8, 4, 128, 1024)) > 0
    # pack: bad dims, null pointers, alignment, a buffer too small
    assert lib.neat_lanes_pack(16, 4, neat.dims(8, 4, 200, 400), 128, 1 << 20, None) == neat.NEAT_EINVAL
    assert lib.neat_lanes_pack(None, 4, d, 128, 1 << 30, None) == neat.NEAT_EINVAL
    assert lib.neat_lanes_pack(16, 4, d, 64, 1 << 30, None) == neat.NEAT_EINVAL          # not 128-byte aligned
    assert lib.neat_lanes_pack(16, 10000, d, 128, n - 1, None) == neat.NEAT_ENOMEM
    # forward: an empty population is a no-op; null pointers and stage sizes are checked
    assert lib.neat_forward_lanes(None, 0, d, None, None, 0, None) == neat.NEAT_OK
    assert lib.neat_forward_lanes(None, 4, d, 16, 16, 0, None) == neat.NEAT_EINVAL
    assert lib.neat_forward_lanes(128, 4, d, None, 16, 0, None) == neat.NEAT_EINVAL      # I > 0 without inputs
    assert lib.neat_forward_lanes(128, 4, neat.dims(8, 4, 129, 200), 16, 16, 0, None) == neat.NEAT_EINVAL
    assert lib.neat_forward_lanes_steps(128, 4, d, 16, 27, 16, 8, -1, 0, None, None) == neat.NEAT_EINVAL
    # tune: the output pointer, the step count and the pointers are checked before any device call
    import ctypes
    sb = ctypes.c_uint32(0)
    assert lib.neat_lanes_tune(128, 4, d, 16, 108, 16, 32, 4, None, None) == neat.NEAT_EINVAL
    assert lib.neat_lanes_tune(128, 4, d, 16, 108, 16, 32, 0, ctypes.byref(sb), None) == neat.NEAT_EINVAL
    assert lib.neat_lanes_tune(None, 4, d, 16, 108, 16, 32, 4, ctypes.byref(sb), None) == neat.NEAT_EINVAL
    assert lib.neat_lanes_tune(64, 4, d, 16, 108, 16, 32, 4, ctypes.byref(sb), None) == neat.NEAT_EINVAL  # alignment
