"""GB300-native spin-adapted, density-fitted EA/IP-ADC(n) (n = 2, 3).

The compute path is the CUDA library ``_build/libadc.so`` (C ABI declared in
``include/adc.h``); this package only marshals arguments to it.  There is no
CPU fallback: if the library is missing, importing the binding raises.
"""
from ._lib import (ADC, ADCBatch, ADCUnrestricted, build_library, library_path, load_library,  # noqa: F401
                   mlp_loss_grad, mlp_nweights, mlp_train, spectrum)

__all__ = ["ADC", "ADCBatch", "ADCUnrestricted", "build_library", "library_path", "load_library", "mlp_loss_grad", "mlp_nweights",
           "mlp_train", "spectrum"]
