"""The default launch shape (fire_default_kernel, the rule fire_init applies)
is a host computation; these CPU tests pin it on the meshes of the
benchmark configurations for a 152-SM GB300 and check its rule on a sweep of
mesh sizes: the tallest strips that keep enough waves of resident CTAs, and
tiles only where even one-cell strips fill under a quarter wave."""
import pytest

import paper_1102_1343_gb300 as pkg

SMS = 152
WARP, MARCH, TILE = pkg.FIRE_KERNEL_WARP, pkg.FIRE_KERNEL_MARCH, pkg.FIRE_KERNEL_TILE


@pytest.fixture(scope="module")
def lib():
    from paper_1102_1343_gb300 import build
    build.build()
    return pkg.load_library()


def cdiv(a, b):
    return -(-a // b)


def ctas(variant, kx, ky, nxa, nya, sr):
    nx, ny = nxa * sr, nya * sr
    if variant == WARP:
        return cdiv(cdiv(nx, kx * sr), 4) * cdiv(ny, ky * sr)
    return cdiv(nx, kx * sr) * cdiv(ny, ky * sr)


@pytest.mark.parametrize("prec,nxa,want", [
    ("fp32", 820, (WARP, 6, 16)),   # 8200^2: 3.99 waves of 60x160 warp strips
    ("fp32", 200, (WARP, 6, 1)),    # 2000^2: ten-row strips
    ("fp32", 10, (TILE, 1, 1)),     # 100^2: one-cell tiles
    ("fp64", 820, (MARCH, 24, 6)),  # 8200^2 FP64: 240x60 marching strips
    ("fp64", 200, (MARCH, 24, 2)),
    ("fp64", 10, (TILE, 1, 1)),
])
def test_benchmark_meshes(lib, prec, nxa, want):
    assert pkg.fire_default_kernel(prec, nxa, nxa, 10, 10, SMS) == want


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_rule_over_mesh_sizes(lib, prec):
    slots, waves2, ky_max = (3 * SMS, 7, 16) if prec == "fp32" else (2 * SMS, 5, 6)
    strip = WARP if prec == "fp32" else MARCH
    for nxa in (12, 25, 51, 80, 133, 200, 347, 512, 820, 1300):
        for nya in (nxa, max(1, nxa // 3), 2 * nxa):
            v, kx, ky = pkg.fire_default_kernel(prec, nxa, nya, 10, 10, SMS)
            one_cell = ctas(strip, 6 if prec == "fp32" else min(24, nxa), 1, nxa, nya, 10)
            if 4 * one_cell < slots:
                assert (v, kx, ky) == (TILE, 1, 1), (nxa, nya)
                continue
            assert v == strip and 1 <= ky <= min(ky_max, nya), (nxa, nya, v, ky)
            assert ky == 1 or 2 * ctas(v, kx, ky, nxa, nya, 10) >= waves2 * slots
            if ky < min(ky_max, nya):
                assert 2 * ctas(v, kx, ky + 1, nxa, nya, 10) < waves2 * slots, (nxa, nya, ky)


def test_large_refinement_and_bad_arguments(lib):
    # refinement 40: too wide for warp strips (<= 30), marching strips of 6 cells
    assert pkg.fire_default_kernel("fp32", 100, 100, 40, 40, SMS) == (MARCH, 6, 1)
    assert pkg.fire_default_kernel("fp64", 100, 100, 40, 40, SMS) == (MARCH, 6, 1)
    # refinement 130: too wide for marching strips (<= 124) -> 2-D tiles of one cell
    assert pkg.fire_default_kernel("fp32", 20, 20, 130, 130, SMS) == (TILE, 1, 1)
    with pytest.raises(pkg.FireError):
        pkg.fire_default_kernel("fp32", 0, 10, 10, 10, SMS)
    with pytest.raises(pkg.FireError):
        pkg.fire_default_kernel(7, 10, 10, 10, 10, SMS)


def test_32bit_offset_limit(lib):
    """The warp kernels' 32-bit offsets take meshes of up to 2^31 - 1 nodes:
    46340^2 = 2,147,395,600 nodes still gets the warp kernel in FP32, 46400 x
    46340 = 2,150,176,000 the marching strips (64-bit offsets)."""
    assert 46340 * 46340 <= 2**31 - 1 < 46400 * 46340
    assert pkg.fire_default_kernel("fp32", 4634, 4634, 10, 10, SMS)[0] == WARP
    assert pkg.fire_default_kernel("fp32", 4640, 4634, 10, 10, SMS)[0] == MARCH
    assert pkg.fire_default_kernel("fp64", 4640, 4634, 10, 10, SMS)[0] == MARCH
