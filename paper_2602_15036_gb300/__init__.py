"""GB300-native SOCS lithography imaging: aerial images, resist and ILT gradients.

The compute runs in liblitho.so (hand-written CUDA for sm_103a behind the C ABI
of include/litho.h); this package is its Python binding (`litho`) and the
in-tree build step (`build`).
"""
from . import litho  # noqa: F401
from .litho import (Kernels, LithoError, litho_aerial, litho_aerial_host, litho_aerial_resist,  # noqa: F401
                    litho_aerial_host_workspace_size, litho_aerial_workspace_size, litho_ilt_grad,
                    litho_ilt_workspace_size, litho_make_kernels, litho_contours, litho_epe, litho_epe_batch, litho_epe_through_focus,
                    litho_rasterize, litho_intensity_vjp, litho_ai_inputs, litho_print_images, litho_tcc_kernels_host, litho_resist, litho_upload_kernels, make_optics)
