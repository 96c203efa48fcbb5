"""Failure detection on the GPU without a fault: a bounded in-kernel wait that
runs out must leave QSVM_ERR_TIMEOUT in the device status word and a usable
context (the next Gram still matches the oracle)."""
import numpy as np
import pytest

from paper_2405_02630_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    assert qsvm.qsvm_device_status(clear=True) == 0
    qsvm.qsvm_selftest_wait_timeout(50_000_000)  # 50 ms on a barrier nothing completes
    torch.cuda.synchronize()
    assert qsvm.qsvm_device_status(clear=True) == qsvm.QSVM_ERR_TIMEOUT
    assert qsvm.qsvm_device_status(clear=False) == 0
    X = inputs.uniform_features(20, 12, 4)
    K, _ = qsvm.gram(torch.from_numpy(X).cuda(), 2, "fp32_split")
    Ko, _ = oracle.mps_gram(X, 2)
    assert np.max(np.abs(K.cpu().numpy() - Ko)) <= 1e-6
    with pytest.raises(qsvm.QsvmError):
        qsvm.qsvm_selftest_wait_timeout(10)
