"""GB300-native QED particle step of the extended PIC scheme of Gonoskov et al.
(arXiv:1412.6426): CUDA kernels for sm_103a behind the C ABI of include/qed.h."""
from . import qed  # noqa: F401
