"""GB300-native fused forward/adjoint simulator for quantum machine learning circuits."""
