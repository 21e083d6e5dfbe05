"""Host-side checks of the torch.autograd binding (no GPU needed)."""
import pytest


def test_autograd_module_imports_and_validates():
    torch = pytest.importorskip("torch")
    from paper_1908_04279_gb300 import autograd as AG
    assert issubclass(AG._MicroSteps, torch.autograd.Function)
    with pytest.raises(ValueError):
        AG.micro_steps(None, None, None, 0.5, 1.0, observable="energy")
