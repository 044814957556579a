"""GB300-native batched three-phase Z-bus power flow."""
