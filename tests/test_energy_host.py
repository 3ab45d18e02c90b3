"""The tuner's energy observer on the CPU, against a fake NVML.

The observer only reads the device's total energy counter (millijoules) through
NVML, opened at run time.  Here a small stand-in library, compiled by the test,
exports the four NVML entry points the observer uses: its counter advances by a
fixed step per read and per device, so the values the library reports can be
checked exactly.  No GPU and no real NVML are involved.
"""
import ctypes
import shutil
import subprocess

import pytest

FAKE_NVML = r"""
typedef struct dev { unsigned int idx; unsigned long long mj; } dev;
static dev devs[2] = {{0, 1000000ull}, {1, 5000000ull}};
int nvmlInit_v2(void) { return 0; }
int nvmlDeviceGetHandleByIndex_v2(unsigned int i, dev **d) { if (i > 1) return 2; *d = &devs[i]; return 0; }
int nvmlDeviceGetHandleByPciBusId_v2(const char *bus, dev **d) { (void)bus; *d = &devs[0]; return 0; }
int nvmlDeviceGetTotalEnergyConsumption(dev *d, unsigned long long *e) {
    d->mj += 1500ull * (d->idx + 1);   /* 1.5 J per read on device 0, 3 J on device 1 */
    *e = d->mj;
    return 0;
}
"""


@pytest.fixture(scope="module")
def kt_fake(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("nvml")
    src, so = d / "fake_nvml.c", d / "libfake_nvml.so"
    src.write_text(FAKE_NVML)
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-o", str(so), str(src)], check=True)
    from paper_2608_21227_gb300 import _build

    _build.build()
    from paper_2608_21227_gb300 import kt

    kt.energy_open(str(so))
    return kt


def test_counter_read_by_index(kt_fake):
    kt = kt_fake
    a = kt.energy_read(index=0)
    b = kt.energy_read(index=0)
    assert b - a == 1500
    c = kt.energy_read(index=1)
    d = kt.energy_read(index=1)
    assert d - c == 3000 and c > 5000000


def test_unknown_device_and_no_cuda(kt_fake):
    kt = kt_fake
    from paper_2608_21227_gb300 import nla

    with pytest.raises(nla.NLAError) as ei:
        kt.energy_read(index=7)
    assert ei.value.status == 1  # NLA_ERR_ARG: NVML knows no such device
    try:
        import torch

        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        # the current-device read needs a CUDA device to find its PCI bus id
        with pytest.raises(nla.NLAError) as ei:
            kt.energy_read()
        assert ei.value.status == 2  # NLA_ERR_CUDA


def test_missing_library_is_unsupported(kt_fake, tmp_path):
    kt = kt_fake
    from paper_2608_21227_gb300 import nla

    with pytest.raises(nla.NLAError) as ei:
        kt.energy_open(str(tmp_path / "no_such_nvml.so"))
    assert ei.value.status == 7  # NLA_ERR_UNSUPPORTED
